"""The sampler's table-driven FP64 exponential against the host libm exp
(numpy): within 2 ulp on a dense sweep of [-700, 700], exact powers of two
at t = k ln 2 multiples, and the library fallback outside the range (inf, 0,
NaN)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _ulp_err(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


def test_exp_dense_sweep():
    from paper_1607_00693_gb300 import api
    rng = np.random.default_rng(11)
    t = np.concatenate([np.linspace(-700, 700, 400001), rng.uniform(-30, 30, 200000),
                        rng.uniform(-1e-3, 1e-3, 20000), [0.0, -0.0, 1e-300, -1e-300]])
    out = api.stomsfem_selftest_exp(torch.from_numpy(t).to("cuda:0")).cpu().numpy()
    err = _ulp_err(out, np.exp(t))
    assert err.max() <= 2.0, (err.max(), t[err.argmax()])
    # table boundaries: t just either side of j ln2/64 for every j
    j = np.arange(-64 * 20, 64 * 20)
    c = j * (np.log(2.0) / 64)
    tb = np.concatenate([np.nextafter(c, -np.inf), c, np.nextafter(c, np.inf)])
    ob = api.stomsfem_selftest_exp(torch.from_numpy(tb).to("cuda:0")).cpu().numpy()
    assert _ulp_err(ob, np.exp(tb)).max() <= 2.0


def test_exp_outside_range_and_special_values():
    from paper_1607_00693_gb300 import api
    t = np.array([-750.0, 710.0, 800.0, -np.inf, np.inf, np.nan, 700.5, -700.5])
    out = api.stomsfem_selftest_exp(torch.from_numpy(t).to("cuda:0")).cpu().numpy()
    ref = np.exp(t)
    assert out[0] == 0.0 or out[0] == ref[0]
    assert np.isinf(out[1]) and np.isinf(out[2]) and out[3] == 0.0 and np.isinf(out[4])
    assert np.isnan(out[5])
    assert _ulp_err(out[6:], ref[6:]).max() <= 2.0
