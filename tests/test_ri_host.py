"""Random-interpolation set-up that runs on the host (no GPU): the library's
plan (directions, degrees, families) against the oracle's own."""
import numpy as np
import pytest

from paper_1607_00693_gb300 import workloads as W


@pytest.fixture(scope="module")
def orc():
    import oracle
    from oracle import ri
    oracle.build()
    return oracle, ri


@pytest.mark.parametrize("name,eps,nu_max", [("msfem_64", 1e-3, 8), ("msfem_64", 3e-3, 8),
                                             ("msfem_64", 1e-2, 3), ("upscale_1024", 1e-1, 4)])
def test_library_plan_matches_oracle(orc, name, eps, nu_max):
    from paper_1607_00693_gb300.build import build_library
    from paper_1607_00693_gb300 import api
    _, ri = orc
    build_library()
    w = W.workload(name)
    g = api.grid(w["nf"], w["nc"], w["f"])
    fam, ids, nu, nfam, npts = api.stomsfem_ri_plan(g, api.field_from_dict(w["field"]), eps, nu_max)
    fo, keys, rep, dims = ri.families(w["nf"], w["nc"], w["field"], eps, nu_max)
    np.testing.assert_array_equal(fam, fo)
    assert nfam == len(keys)
    assert npts == sum(int(np.prod([k[2] + 1 for k in key])) for key in keys)
    for c, d in enumerate(dims):
        assert list(ids[c, :len(d)]) == [v for (_, _, _, v) in d] and np.all(ids[c, len(d):] == -1)
        assert list(nu[c, :len(d)]) == [n for (_, _, n, _) in d] and np.all(nu[c, len(d):] == 0)


def test_library_plan_rejects_oversized_grids(orc):
    from paper_1607_00693_gb300.build import build_library
    from paper_1607_00693_gb300 import api, _lib
    build_library()
    w = W.workload("contrast_2048")
    g = api.grid(w["nf"], w["nc"], w["f"])
    with pytest.raises(_lib.StomsfemError):
        api.stomsfem_ri_plan(g, api.field_from_dict(w["field"]), 1e-3, 8)
    w = W.workload("msfem_64")
    g = api.grid(w["nf"], w["nc"], w["f"])
    for bad in (dict(eps=0.0, nu_max=8), dict(eps=1e-3, nu_max=0), dict(eps=1e-3, nu_max=9)):
        with pytest.raises(_lib.StomsfemError):
            api.stomsfem_ri_plan(g, api.field_from_dict(w["field"]), bad["eps"], bad["nu_max"])


def test_library_plan_matches_oracle_sigmoid_field(orc):
    """The sigmoid transform's strength |L gain| / 4 exp(-d^2/w^2) (a field
    with contrast 10 on the 64^2 / 8^2 grid): same families, directions and
    degrees as the oracle."""
    import math
    from paper_1607_00693_gb300.build import build_library
    from paper_1607_00693_gb300 import api
    _, ri = orc
    build_library()
    fld = dict(kind=1, nbx=4, nby=4, width=0.1, scale=1.0, contrast_log=math.log(10.0), gain=1.0)
    g = api.grid(64, 8, 1.0)
    fam, ids, nu, nfam, npts = api.stomsfem_ri_plan(g, api.field_from_dict(fld), 1e-3, 6)
    fo, keys, rep, dims = ri.families(64, 8, fld, 1e-3, 6)
    np.testing.assert_array_equal(fam, fo)
    assert nfam == len(keys) == 36
    for c, d in enumerate(dims):
        assert list(ids[c, :len(d)]) == [v for (_, _, _, v) in d]
        assert list(nu[c, :len(d)]) == [n for (_, _, n, _) in d]


def test_degree_rule_golden(orc):
    """Hand-worked degrees of tests/golden/ri_degree_rule.txt: the oracle's
    rule, and the library's plan for one bump centred in the only cell
    (influence g = scale)."""
    import os
    from paper_1607_00693_gb300.build import build_library
    from paper_1607_00693_gb300 import api
    _, ri = orc
    build_library()
    rows = [line.split() for line in open(os.path.join(os.path.dirname(__file__), "golden", "ri_degree_rule.txt"))
            if line.strip() and not line.startswith("#")]
    for g_s, eps_s, nm_s, nu_s in rows:
        g, eps, nm, nu = float(g_s), float(eps_s), int(nm_s), int(nu_s)
        assert ri.choose_nu(g, eps, nm) == nu, (g, eps, nm)
        fld = dict(kind=0, nbx=1, nby=1, width=0.3, scale=g, contrast_log=0.0, gain=1.0)
        _, ids, nus, _, npts = api.stomsfem_ri_plan(api.grid(8, 1, 1.0), api.field_from_dict(fld), eps, nm)
        if nu == 0:
            assert np.all(ids[0] == -1) and npts == 1
        else:
            assert ids[0, 0] == 0 and nus[0, 0] == nu and np.all(ids[0, 1:] == -1), (g, eps, nm)
            assert npts == nu + 1
