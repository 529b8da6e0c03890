"""A bounded device wait that runs out: the kernel waits on an mbarrier
nothing arrives at, gives up after its iteration limit, reports
STOMSFEM_ETIMEOUT in a status word, and the context stays usable (a normal
computation runs correctly right after)."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_wait_runs_out_and_context_survives(orc):
    from paper_1607_00693_gb300 import api, _lib as L
    assert api.stomsfem_selftest_wait_timeout(2000) == L.ETIMEOUT
    assert api.stomsfem_selftest_wait_timeout(1) == L.ETIMEOUT
    # the device still computes: one small upscale against the oracle
    import numpy as np
    g = api.grid(32, 4)
    rng = np.random.default_rng(7)
    a = np.exp(rng.normal(size=(2, 32, 32)))
    Ke_ref, be_ref = orc.upscale(32, 4, 1.0, a)
    dev = torch.device("cuda:0")
    at = torch.tensor(a, device=dev)
    Ke = torch.empty((2, 16, 10), dtype=torch.float64, device=dev)
    be = torch.empty((2, 16, 4), dtype=torch.float64, device=dev)
    api.stomsfem_upscale(g, at, Ke, be)
    torch.cuda.synchronize()
    assert np.abs(Ke.cpu().numpy() - Ke_ref).max() <= 1e-11 * np.abs(Ke_ref).max()
