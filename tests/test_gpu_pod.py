"""Reduced-basis (POD) path on the GPU vs the FP64 POD oracle.

Offline: the GPU builds the per-cell basis from its own FP64 snapshots; the
oracle builds its basis from its own snapshots; ranks are pinned to the
oracle's so both use the same subspace dimension.  Online: K_e and b_e
after FP64 refinement within 1e-10 of the oracle's reduced-basis K_e (the
result depends on the subspace only); without refinement (BF16 tensor-core
reduced matrices) within 5e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"


@pytest.fixture(scope="module")
def setup():
    import oracle
    from oracle import pod
    from paper_1607_00693_gb300.build import build_library
    oracle.build()
    build_library()
    w = W.workload("pod_64")
    nf, nc = w["nf"], w["nc"]
    Ns = 40
    xi = W.draw_xi(w["field"], Ns, w["train_seed"])
    a_tr = oracle.sample_coef(nf, w["field"], xi)
    _, _, phi_o = oracle.upscale(nf, nc, w["f"], a_tr, want_phi=True)
    models = pod.build(nf, nc, phi_o, a_tr, tol=1e-6, max_rank=27)
    ranks = [m["rank"] for m in models]
    g = api.grid(nf, nc, w["f"])
    a_t = torch.from_numpy(a_tr).to(DEV)
    rho = nf // nc
    Ke = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=DEV)
    phi = torch.empty((Ns, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a_t, Ke, be, phi=phi)
    h, rk = api.stomsfem_pod_build(g, phi, a_t, ranks=ranks)
    hfree, rk_free = api.stomsfem_pod_build(g, phi, a_t, tol=1e-6, max_rank=27)
    xt = W.draw_xi(w["field"], 37, w["seed"])
    a_te = oracle.sample_coef(nf, w["field"], xt)
    yield dict(oracle=oracle, pod=pod, w=w, g=g, models=models, ranks=ranks, h=h, rk=rk,
               rk_free=rk_free, hfree=hfree, a_te=a_te, nf=nf, nc=nc)
    api.stomsfem_pod_destroy(h)
    api.stomsfem_pod_destroy(hfree)


def _gpu(setup, refine, handle=None):
    g, nc = setup["g"], setup["nc"]
    a = torch.from_numpy(setup["a_te"]).to(DEV)
    S = a.shape[0]
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=DEV)
    st = torch.full((S, nc * nc), 9, dtype=torch.int32, device=DEV)
    api.stomsfem_pod_upscale(handle or setup["h"], g, a, Ke, be, refine_iters=refine, unit_status=st)
    torch.cuda.synchronize()
    return Ke.cpu().numpy(), be.cpu().numpy(), st.cpu().numpy()


def _rel(x, y):
    return float(np.max(np.linalg.norm(x - y, axis=-1) / np.linalg.norm(y, axis=-1)))


def test_pod_ranks(setup):
    assert setup["rk"] == setup["ranks"]
    # the GPU's own truncation agrees with the oracle's up to ties at the threshold
    assert max(abs(a - b) for a, b in zip(setup["rk_free"], setup["ranks"])) <= 1


def test_pod_eigenvalues(setup):
    lam = api.stomsfem_pod_eigenvalues(setup["h"], setup["g"])
    for cell in (0, 9, 27, 63):
        lo = setup["models"][cell]["lam"]
        keep = lo / lo[0] > 1e-8
        np.testing.assert_allclose(lam[cell][keep], lo[keep], rtol=1e-8)


def test_pod_refined_matches_oracle(setup):
    Ko, bo = setup["pod"].upscale(setup["models"], setup["nf"], setup["nc"], 1.0, setup["a_te"])
    Kg, bg, st = _gpu(setup, refine=8)
    assert np.all(st == 0)
    assert _rel(Kg, Ko) <= 1e-10
    assert _rel(bg, bo) <= 1e-10
    K = Kg.reshape(-1, 10)
    rows = K[:, 0] + K[:, 1] + K[:, 2] + K[:, 3]
    assert np.max(np.abs(rows)) <= 1e-10 * np.max(np.abs(K))


def test_pod_unrefined_tensor_core(setup):
    """Without refinement: one BF16 product per K step (8 significant bits in
    G) within 5e-3 of the oracle's reduced basis; the default BF16 pairs
    (three products, about 16 bits) within 1e-4 and closer than one pass."""
    Ko, bo = setup["pod"].upscale(setup["models"], setup["nf"], setup["nc"], 1.0, setup["a_te"])
    api.stomsfem_pod_set_gemm_split(setup["h"], 0)
    try:
        K1, b1, st1 = _gpu(setup, refine=0)
    finally:
        api.stomsfem_pod_set_gemm_split(setup["h"], 1)
    Kg, bg, st = _gpu(setup, refine=0)
    assert np.all(st == 0) and np.all(st1 == 0)
    assert _rel(K1, Ko) <= 5e-3
    assert _rel(b1, bo) <= 5e-3
    print("H/h = 8 POD unrefined: one pass %.3e, split %.3e" % (_rel(K1, Ko), _rel(Kg, Ko)))
    assert _rel(Kg, Ko) <= 1e-4
    assert _rel(bg, bo) <= 1e-4
    assert _rel(Kg, Ko) < _rel(K1, Ko)


def test_pod_vs_plain_msfem(setup):
    """The reduced model stays close to the plain upscaler (truncation at
    1e-6 relative energy)."""
    Kp, bp = setup["oracle"].upscale(setup["nf"], setup["nc"], 1.0, setup["a_te"])
    Kg, _, _ = _gpu(setup, refine=8)
    assert _rel(Kg, Kp) <= 1e-4


def test_pod_checkpoint_roundtrip(setup):
    """A saved and reloaded offline stage gives bit-identical online results
    (refined and unrefined) and the same ranks and eigenvalues."""
    data = api.stomsfem_pod_save(setup["h"])
    h2 = api.stomsfem_pod_load(data)
    try:
        for refine in (0, 2):
            K1, b1, s1 = _gpu(setup, refine)
            K2, b2, s2 = _gpu(setup, refine, handle=h2)
            assert np.array_equal(K1, K2) and np.array_equal(b1, b2) and np.array_equal(s1, s2)
        g = setup["g"]
        assert np.array_equal(api.stomsfem_pod_eigenvalues(h2, g), api.stomsfem_pod_eigenvalues(setup["h"], g))
        assert api.stomsfem_pod_save(h2) == data
    finally:
        api.stomsfem_pod_destroy(h2)
