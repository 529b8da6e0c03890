"""Surrogate set-up logic that runs on the host (no GPU): the library's
local-variable and family tables against the oracle's own implementation."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W


@pytest.mark.parametrize("name,tau", [("surrogate_64", 1e-6), ("surrogate_64", 1e-4), ("msfem_64", 1e-2)])
def test_local_vars_match_oracle(name, tau):
    from paper_1607_00693_gb300.build import build_library
    from paper_1607_00693_gb300 import api
    from oracle import surrogate as S
    build_library()
    w = W.workload(name)
    g = api.grid(w["nf"], w["nc"], w["f"])
    k, ids, fam, nfam = api.stomsfem_local_vars(g, api.field_from_dict(w["field"]), tau)
    ko, idso, famo, nfamo = S.local_vars(w["nf"], w["nc"], w["field"], tau)
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(ids, idso)
    np.testing.assert_array_equal(fam, famo)
    assert nfam == nfamo


def test_local_vars_surrogate_64_sizes():
    """At tau = 1e-6 every cell of the surrogate workload sees 4..9 local
    variables (the K_m of Eq. MsFEB2), grouped into 36 patch families."""
    from oracle import surrogate as S
    w = W.workload("surrogate_64")
    k, ids, fam, nfam = S.local_vars(w["nf"], w["nc"], w["field"], 1e-6)
    assert k.min() == 4 and k.max() == 9 and nfam == 36
    # every family's cells have the same count; ids are distinct within a cell
    for f in range(nfam):
        assert len(set(k[fam == f])) == 1
    for c in range(len(k)):
        v = ids[c, :k[c]]
        assert len(set(v)) == len(v) and np.all(ids[c, k[c]:] == -1)
