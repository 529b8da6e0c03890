"""The surrogate's error indicator on the GPU, flag by flag against the
oracle's restatement of the rule (oracle/surrogate.py: indicator).

The network is made to output chosen matrices: the last layer's weights are
zero, so every unit of a family gets that family's output bias y exactly,
and K = abar (K_ref + P y) with P the zero-row-sum projector.  Families are
given y = alpha K_ref (both corner energies (1 + alpha) abar: a sweep across
the harmonic lower bound, just inside and outside the upper bound) or
y = -beta v_h v_h^T (v_h = (1, -1, 1, -1): energies unchanged, indefinite
exactly when beta > 1/6), and a training box of [-0.9, 0.9] for the used
inputs, so that the range test fires on the units with some |xi_j| above
0.918 (1% margin).  The box and weights enter through a checkpoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1607_00693_gb300 import api
from paper_1607_00693_gb300 import workloads as W

DEV = "cuda:0"
DELTA = 0.02
MARGIN = 0.01


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1607_00693_gb300.build import build_library
    build_library()


def _family_outputs(nfam):
    """y (16) per family and the role of each family."""
    from oracle import surrogate as S
    kref = S.KREF_PACKED
    vh = np.array([1.0, -1.0, 1.0, -1.0])
    hour = S.pack_upper_sym(np.outer(vh, vh))
    ys = np.zeros((nfam, 16))
    alphas = list(np.linspace(-0.30, -0.01, 12)) + [DELTA + 0.004, DELTA + 0.02, 0.1, DELTA - 0.004,
                                                    DELTA - 0.01, 0.0]
    betas = [0.12, 0.15, 0.18, 0.22, 0.3]
    for f in range(nfam):
        if f < len(alphas):
            ys[f, :10] = alphas[f] * kref
        elif f < len(alphas) + len(betas):
            ys[f, :10] = -betas[f - len(alphas)] * hour
        else:
            ys[f, :10] = 0.0
    return ys


def test_indicator_flags_match_oracle(orc):
    from oracle import surrogate as S
    w = W.workload("surrogate_64")
    nf, nc = w["nf"], w["nc"]
    rho, H = nf // nc, 1.0 / nc
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    k, ids, fam, nfam = S.local_vars(nf, nc, w["field"], 1e-6)
    weights = api.xavier_weights(nfam, 2)
    ys = _family_outputs(nfam).astype(np.float32)
    o_w4, o_b4 = 2 * (128 * 128 + 128) + 128 * 16 + 128, 2 * (128 * 128 + 128) + 128 * 16 + 128 + 16 * 128
    weights[:, o_w4:o_b4] = 0.0
    weights[:, o_b4:o_b4 + 16] = ys
    h, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, weights)
    data = bytearray(api.stomsfem_surrogate_save(h))
    api.stomsfem_surrogate_destroy(h)
    box = np.zeros((nfam, 16, 2), dtype=np.float32)
    for c in range(nc * nc):
        box[fam[c], :k[c], 0] = -0.9
        box[fam[c], :k[c], 1] = 0.9
    nb = box.size * 4
    data[-nb:] = box.tobytes()
    h, _ = api.stomsfem_surrogate_load(bytes(data))
    try:
        S_ = 200
        xi = W.draw_xi(w["field"], S_, 31)
        a = orc.sample_coef(nf, w["field"], xi)
        xt = torch.from_numpy(xi).to(DEV)
        at = torch.from_numpy(a).to(DEV)
        Ke = torch.empty((S_, nc * nc, 10), dtype=torch.float64, device=DEV)
        be = torch.empty((S_, nc * nc, 4), dtype=torch.float64, device=DEV)
        fb = torch.empty((S_, nc * nc), dtype=torch.uint8, device=DEV)
        api.stomsfem_surrogate_infer(h, g, xt, at, Ke, be, fb, delta=DELTA)
        torch.cuda.synchronize()
        flags = fb.cpu().numpy()
    finally:
        api.stomsfem_surrogate_destroy(h)
    from oracle import mlp
    P = mlp.zero_row_sum_projector()
    kref = S.KREF_PACKED
    counts = {"none": 0, "range": 0, "energy_low": 0, "energy_high": 0, "pd": 0}
    ambiguous = mismatched = 0
    for s in range(S_):
        for c in range(nc * nc):
            f = fam[c]
            x = np.zeros(16)
            x[:k[c]] = xi[s, ids[c, :k[c]]].astype(np.float32)
            blk = a[s, (c // nc) * rho:(c // nc + 1) * rho, (c % nc) * rho:(c % nc + 1) * rho]
            abar, ahar = blk.mean(), 1.0 / np.mean(1.0 / blk)
            Kp = abar * (kref + P @ ys[f, :10].astype(np.float64))
            r = S.indicator(x, box[f], MARGIN, Kp, abar, ahar, DELTA)
            ex, ey = S.energy_values(Kp)
            # a decision within 1e-5 of a bound is left out: the two sides
            # evaluate K and the harmonic mean with different roundings
            near = min(abs(e - b) / b for e in (ex, ey) for b in (ahar * (1 - DELTA), abar * (1 + DELTA)))
            if near < 1e-5:
                ambiguous += 1
                continue
            want = any(r.values())
            if bool(flags[s, c]) != want:
                mismatched += 1
            reasons = [n for n, v in r.items() if v]
            if not reasons:
                counts["none"] += 1
            elif reasons == ["range"]:
                counts["range"] += 1
            elif reasons == ["pd"]:
                counts["pd"] += 1
            elif reasons == ["energy"]:
                counts["energy_low" if max(ex, ey) < abar else "energy_high"] += 1
    print("indicator cases", counts, "ambiguous", ambiguous)
    assert mismatched == 0
    assert ambiguous <= 5
    # every bound has units that trip it alone, and units pass every test
    for key, n in counts.items():
        assert n >= 20, (key, counts)


def _bias_only_handle(g, fld, nfam, ys, box_of_fam):
    """A surrogate whose network outputs exactly ys[f] for family f (zero
    last-layer weights, the outputs in the bias), with a given input box."""
    weights = api.xavier_weights(nfam, 3)
    o_w4, o_b4 = 2 * (128 * 128 + 128) + 128 * 16 + 128, 2 * (128 * 128 + 128) + 128 * 16 + 128 + 16 * 128
    weights[:, o_w4:o_b4] = 0.0
    weights[:, o_b4:o_b4 + 16] = ys.astype(np.float32)
    h, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, weights)
    data = bytearray(api.stomsfem_surrogate_save(h))
    api.stomsfem_surrogate_destroy(h)
    nb = box_of_fam.size * 4
    data[-nb:] = box_of_fam.astype(np.float32).tobytes()
    h, _ = api.stomsfem_surrogate_load(bytes(data))
    return h


def test_ensemble_flags_and_fallback(orc):
    """Two networks with known outputs: the first K = abar K_ref on every
    unit (accepted by every rule), the partner K = abar (1 + eps_f) K_ref
    with eps_f spread over [0, 0.1] by family, so that the two differ by
    exactly eps_f relative.  With tol = 0.05 the flags are 2 on the
    families the oracle's rule (ensemble_disagrees) flags and 0 elsewhere;
    the flagged units hold the plain FP64 upscaler's K_e, the others
    abar K_ref; without the partner nothing falls back; a partner of other
    families is refused."""
    from oracle import surrogate as S
    w = W.workload("surrogate_64")
    nf, nc = w["nf"], w["nc"]
    rho = nf // nc
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    k, ids, fam, nfam = S.local_vars(nf, nc, w["field"], 1e-6)
    kref = S.KREF_PACKED
    box = np.zeros((nfam, 16, 2))
    box[:, :, 0], box[:, :, 1] = -2.0, 2.0
    eps = np.linspace(0.0, 0.1, nfam)
    eps[np.abs(eps - 0.05) < 2e-3] += 5e-3       # keep every family clear of the threshold
    y1 = np.zeros((nfam, 16))
    y2 = np.zeros((nfam, 16))
    y2[:, :10] = eps[:, None] * kref[None, :]
    h1 = _bias_only_handle(g, fld, nfam, y1, box)
    h2 = _bias_only_handle(g, fld, nfam, y2, box)
    hx, _ = api.stomsfem_surrogate_create(g, fld, 1e-2, api.xavier_weights(
        len(set(S.local_vars(nf, nc, w["field"], 1e-2)[2])), 4))
    try:
        with pytest.raises(Exception):
            api.stomsfem_surrogate_set_partner(h1, hx, 0.05)   # other families (tau 1e-2)
        with pytest.raises(Exception):
            api.stomsfem_surrogate_set_partner(h1, h1, 0.05)
        S_ = 40
        xi = W.draw_xi(w["field"], S_, 33)
        a = orc.sample_coef(nf, w["field"], xi)
        xt = torch.from_numpy(xi).to(DEV)
        at = torch.from_numpy(a).to(DEV)
        Ke = torch.empty((S_, nc * nc, 10), dtype=torch.float64, device=DEV)
        be = torch.empty((S_, nc * nc, 4), dtype=torch.float64, device=DEV)
        fb = torch.empty((S_, nc * nc), dtype=torch.uint8, device=DEV)
        api.stomsfem_surrogate_infer(h1, g, xt, at, Ke, be, fb, delta=DELTA)
        torch.cuda.synchronize()
        assert int(fb.sum().item()) == 0                        # no partner: every unit accepted
        api.stomsfem_surrogate_set_partner(h1, h2, 0.05)
        api.stomsfem_surrogate_infer(h1, g, xt, at, Ke, be, fb, delta=DELTA)
        torch.cuda.synchronize()
        flags, Kg = fb.cpu().numpy(), Ke.cpu().numpy()
        api.stomsfem_surrogate_set_partner(h1, None, 0.0)
        api.stomsfem_surrogate_infer(h1, g, xt, at, Ke, be, fb, delta=DELTA)
        torch.cuda.synchronize()
        assert int(fb.sum().item()) == 0                        # partner removed
    finally:
        for h in (h1, h2, hx):
            api.stomsfem_surrogate_destroy(h)
    Kplain, _ = orc.upscale(nf, nc, w["f"], a)
    n2 = 0
    for s in range(S_):
        for c in range(nc * nc):
            blk = a[s, (c // nc) * rho:(c // nc + 1) * rho, (c % nc) * rho:(c % nc + 1) * rho]
            abar = blk.mean()
            K1, K2 = abar * kref, abar * (1 + eps[fam[c]]) * kref
            want = S.ensemble_disagrees(K1, K2, 0.05)
            assert flags[s, c] == (2 if want else 0), (s, c, eps[fam[c]])
            if want:
                n2 += 1
                np.testing.assert_allclose(Kg[s, c], Kplain[s, c], rtol=1e-11, atol=1e-13)
            else:
                np.testing.assert_allclose(Kg[s, c], K1, rtol=1e-6)
    assert 0.2 * S_ * nc * nc < n2 < 0.8 * S_ * nc * nc
