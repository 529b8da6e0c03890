"""Merge of running Monte Carlo moments (the exchange a multi-GPU run ends
with: each rank's (mean, M2, count) folded into one): the merged moments
of three uneven sample sets equal the oracle's two-pass moments of all the
samples together (Eq. MCestimate), in either merge order; an empty set
leaves the other unchanged; bad arguments are refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api

DEV = "cuda:0"


@pytest.fixture(scope="module")
def lib():
    from paper_1607_00693_gb300.build import build_library
    build_library()


def _moments(u):
    n = u.shape[1]
    mean = torch.zeros(n, dtype=torch.float64, device=DEV)
    m2 = torch.zeros_like(mean)
    cnt = torch.zeros(1, dtype=torch.float64, device=DEV)
    api.stomsfem_mc_moments(u, mean, m2, cnt)
    return mean, m2, cnt


def test_merge_equals_moments_of_the_union(lib, orc):
    r = np.random.default_rng(5)
    n = 1089   # (nc + 1)^2 at nc = 32
    sets = [r.normal(1.0 + k, 0.1 * (k + 1), size=(S, n)) for k, S in enumerate((7, 40, 129))]
    mo, vo = orc.mc_moments(np.concatenate(sets))
    for order in ((0, 1, 2), (2, 0, 1)):
        acc = _moments(torch.from_numpy(sets[order[0]]).to(DEV))
        for k in order[1:]:
            b = _moments(torch.from_numpy(sets[k]).to(DEV))
            api.stomsfem_mc_merge(*acc, *b)
        torch.cuda.synchronize()
        assert acc[2].item() == 176
        np.testing.assert_allclose(acc[0].cpu().numpy(), mo, rtol=1e-13, atol=0)
        np.testing.assert_allclose(acc[1].cpu().numpy() / 176, vo, rtol=1e-10)


def test_merge_with_empty_set(lib):
    u = torch.from_numpy(np.random.default_rng(6).normal(size=(9, 33))).to(DEV)
    acc = _moments(u)
    ref = [t.clone() for t in acc]
    empty = (torch.zeros(33, dtype=torch.float64, device=DEV), torch.zeros(33, dtype=torch.float64, device=DEV),
             torch.zeros(1, dtype=torch.float64, device=DEV))
    api.stomsfem_mc_merge(*acc, *empty)
    torch.cuda.synchronize()
    for x, y in zip(acc, ref):
        assert torch.equal(x, y)
    # merging into an empty set copies the other
    e2 = [t.clone() for t in empty]
    api.stomsfem_mc_merge(*e2, *ref)
    torch.cuda.synchronize()
    for x, y in zip(e2, ref):
        assert torch.allclose(x, y, rtol=1e-15, atol=0)


def test_merge_rejects_bad_arguments(lib):
    from paper_1607_00693_gb300 import _lib as L
    assert L.lib().stomsfem_mc_merge(0, None, None, None, None, None, None, None) == L.EINVAL
    assert L.lib().stomsfem_mc_merge(4, None, None, None, None, None, None, None) == L.EINVAL
