"""Per-l reduced bases (one KL basis for each of phi^1, phi^2, phi^3, the
patch study of Sec. 5.1; phi^4 from the partition of unity) on the GPU
against the FP64 per-l POD oracle (oracle/pod.py: build_cell_per_l,
online_cell_per_l).  The GPU builds its bases from its own FP64 snapshots,
the oracle from its own; ranks are pinned to the oracle's.  Online: K_e and
b_e after FP64 refinement within 1e-10 of the oracle's per-l reduced-basis
result (it depends on the three subspaces only); without refinement (BF16
tensor-core reduced matrices) within 5e-3, as the shared-basis form."""
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
    models = pod.build_per_l(nf, nc, phi_o, a_tr, tol=1e-6, max_rank=9)
    ranks = [list(m["rank"]) for m in models]
    g = api.grid(nf, nc, w["f"])
    a_t = torch.from_numpy(a_tr).to(DEV)
    rho = nf // nc
    Ke = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=DEV)
    be = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=DEV)
    phi = torch.empty((Ns, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=DEV)
    api.stomsfem_upscale(g, a_t, Ke, be, phi=phi)
    h, rk = api.stomsfem_pod_build_per_l(g, phi, a_t, max_rank_per_l=9, ranks=ranks)
    hfree, rk_free = api.stomsfem_pod_build_per_l(g, phi, a_t, tol=1e-6, max_rank_per_l=9)
    xt = W.draw_xi(w["field"], 29, w["seed"] + 1)
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


def test_per_l_ranks_and_eigenvalues(setup):
    assert setup["rk"] == setup["ranks"]
    diff = max(abs(a - b) for ra, rb in zip(setup["rk_free"], setup["ranks"]) for a, b in zip(ra, rb))
    assert diff <= 1  # the GPU's own truncation, up to ties at the threshold
    lam = api.stomsfem_pod_eigenvalues(setup["h"], setup["g"], per_l=True)
    for cell in (0, 9, 27, 63):
        for l in range(3):
            lo = setup["models"][cell]["lam"][l]
            keep = lo / lo[0] > 1e-8
            np.testing.assert_allclose(lam[cell, l][keep], lo[keep], rtol=1e-8)


def test_per_l_refined_matches_oracle(setup):
    Ko, bo = setup["pod"].upscale_per_l(setup["models"], setup["nf"], setup["nc"], 1.0, setup["a_te"])
    Kg, bg, st = _gpu(setup, refine=8)
    assert np.all(st == 0)
    assert _rel(Kg, Ko) <= 1e-10
    assert _rel(bg, bo) <= 1e-10
    K = Kg.reshape(-1, 10)
    rows = K[:, 0] + K[:, 1] + K[:, 2] + K[:, 3]
    assert np.max(np.abs(rows)) <= 1e-10 * np.max(np.abs(K))
    H2 = 1.0 / setup["nc"] ** 2
    assert np.max(np.abs(bg.sum(axis=-1) - H2)) <= 1e-12


def test_per_l_unrefined_tensor_core(setup):
    Ko, bo = setup["pod"].upscale_per_l(setup["models"], setup["nf"], setup["nc"], 1.0, setup["a_te"])
    Kg, bg, st = _gpu(setup, refine=0)
    assert np.all(st == 0)
    assert _rel(Kg, Ko) <= 5e-3
    assert _rel(bg, bo) <= 5e-3


def test_per_l_vs_plain_msfem(setup):
    """Three bases truncated at 1e-6 stay close to the plain upscaler."""
    Kp, _ = setup["oracle"].upscale(setup["nf"], setup["nc"], 1.0, setup["a_te"])
    Kg, _, _ = _gpu(setup, refine=8)
    assert _rel(Kg, Kp) <= 1e-4


def test_per_l_checkpoint_roundtrip(setup):
    data = api.stomsfem_pod_save(setup["h"])
    assert data[:8] == b"STMFPODL"
    h2 = api.stomsfem_pod_load(data)
    try:
        for refine in (0, 2):
            K1, b1, s1 = _gpu(setup, refine)
            K2, b2, s2 = _gpu(setup, refine, handle=h2)
            assert np.array_equal(K1, K2) and np.array_equal(b1, b2) and np.array_equal(s1, s2)
        assert api.stomsfem_pod_save(h2) == data
    finally:
        api.stomsfem_pod_destroy(h2)
