"""Pins for the oracle's estimator (Eqs. 2-7 with the zero-width kernel limit).

Each test checks a property the mathematics fixes, independently of the oracle's own
formulas: one-sample and identical-sample events, invariance under sample and event
permutation, the exact shift from the PE prior, independence of the pixel ids when
all LOS rows are equal, the H0 <-> d_L scaling symmetry, the selection identity
xi = N_found / N_draw when the draw density equals the population, unit
normalisation of the detector-frame population density (which fixes every Jacobian),
the flag rules, and the gradient against central finite differences.
"""
import math

import numpy as np
import pytest

from conftest import smooth_row, tiny_catalogue
from paper_2605_23538_gb300.synth import FIDUCIAL

C_KMS = 299792.458


def _events_from(cat, n_ev, per, rng, pixels):
    """n_ev events of ``per`` samples drawn (with replacement) from catalogue samples."""
    idx = rng.integers(0, len(cat["m1"]), size=(n_ev, per))
    ev = []
    for e in range(n_ev):
        ev.append([(cat["m1"][k], cat["m2"][k], cat["dl"][k], cat["lnpe"][k], rng.choice(pixels))
                   for k in idx[e]])
    return ev


def _inj_from(cat, n, rng):
    k = rng.integers(0, len(cat["inj_m1"]), size=n)
    return [(cat["inj_m1"][i], cat["inj_m2"][i], cat["inj_dl"][i], cat["inj_lnpd"][i]) for i in k]


@pytest.fixture(scope="module")
def small(cat_c1):
    rng = np.random.default_rng(5)
    row = smooth_row(257)
    rows = np.stack([row, row * np.float32(1.5), row * np.float32(0.5)])
    rows = rows / rows.mean(axis=0).sum() * row.sum()  # any positive rows will do
    ev = _events_from(cat_c1, 4, 40, rng, [0, 1, 2])
    inj = _inj_from(cat_c1, 300, rng)
    return tiny_catalogue(rows, ev, inj, n_draw=1000.0)


def test_single_sample_event_equals_its_weight(orc, cat_c1):
    row = smooth_row(129)
    rows = np.stack([row, row])
    s = (cat_c1["m1"][3], cat_c1["m2"][3], cat_c1["dl"][3], cat_c1["lnpe"][3])
    inj = [(cat_c1["inj_m1"][i], cat_c1["inj_m2"][i], cat_c1["inj_dl"][i], cat_c1["inj_lnpd"][i])
           for i in range(50)]
    cat = tiny_catalogue(rows, [[(*s, 1)]], inj, 100.0)
    out = orc.loglik(cat, FIDUCIAL, neff_min_event=1.0)
    lw = orc.ln_w_row(FIDUCIAL, [s[0]], [s[1]], [s[2]], [s[3]], row, 2.0)[0]
    assert np.isfinite(lw)
    assert out["lnL_event"][0, 0] == pytest.approx(lw, abs=1e-12)
    assert out["neff_event"][0, 0] == pytest.approx(1.0, abs=1e-12)


def test_identical_samples(orc, cat_c1):
    row = smooth_row(129)
    s = (cat_c1["m1"][7], cat_c1["m2"][7], cat_c1["dl"][7], cat_c1["lnpe"][7], 0)
    inj = [(cat_c1["inj_m1"][i], cat_c1["inj_m2"][i], cat_c1["inj_dl"][i], cat_c1["inj_lnpd"][i])
           for i in range(50)]
    cat1 = tiny_catalogue([row], [[s]], inj, 100.0)
    cat9 = tiny_catalogue([row], [[s] * 9], inj, 100.0)
    a = orc.loglik(cat1, FIDUCIAL, neff_min_event=0.0)
    b = orc.loglik(cat9, FIDUCIAL, neff_min_event=0.0)
    assert b["lnL_event"][0, 0] == pytest.approx(a["lnL_event"][0, 0], abs=1e-12)
    assert b["neff_event"][0, 0] == pytest.approx(9.0, rel=1e-13)


def test_sample_and_event_permutation(orc, small):
    rng = np.random.default_rng(11)
    base = orc.loglik(small, FIDUCIAL, neff_min_event=0.0)
    off = small["offsets"]
    perm_ev = rng.permutation(len(off) - 1)
    pieces = []
    for e in perm_ev:
        idx = np.arange(off[e], off[e + 1])
        pieces.append(rng.permutation(idx))
    sel = np.concatenate(pieces)
    cat = dict(small)
    counts = np.diff(off)[perm_ev]
    cat["offsets"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    for k in ("m1", "m2", "dl", "lnpe", "pix"):
        cat[k] = small[k][sel]
    ip = rng.permutation(len(small["inj_m1"]))
    for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
        cat[k] = small[k][ip]
    got = orc.loglik(cat, FIDUCIAL, neff_min_event=0.0)
    np.testing.assert_allclose(got["lnL_event"][0], base["lnL_event"][0][perm_ev], rtol=0, atol=1e-12)
    assert got["ln_xi"][0] == pytest.approx(base["ln_xi"][0], abs=1e-12)
    assert got["lnL_total"][0] == pytest.approx(base["lnL_total"][0], abs=1e-10)


def test_pe_prior_shift(orc, small):
    c = 0.8125  # exactly representable, so ln pi + c is exact in float32 for these magnitudes
    cat = dict(small)
    cat["lnpe"] = (small["lnpe"].astype(np.float64) + c).astype(np.float32)
    shift = cat["lnpe"].astype(np.float64) - small["lnpe"].astype(np.float64)
    assert np.allclose(shift, c, atol=0)
    a = orc.loglik(small, FIDUCIAL, neff_min_event=0.0)
    b = orc.loglik(cat, FIDUCIAL, neff_min_event=0.0)
    np.testing.assert_allclose(b["lnL_event"] - a["lnL_event"], -c, atol=1e-12)
    assert b["ln_xi"][0] == a["ln_xi"][0]
    cat2 = dict(small)
    cat2["inj_lnpd"] = (small["inj_lnpd"].astype(np.float64) + c).astype(np.float32)
    d = orc.loglik(cat2, FIDUCIAL, neff_min_event=0.0)
    assert d["ln_xi"][0] - a["ln_xi"][0] == pytest.approx(-c, abs=1e-12)
    n_ev = len(small["offsets"]) - 1
    assert d["lnL_total"][0] - a["lnL_total"][0] == pytest.approx(n_ev * c, abs=1e-10)


def test_equal_rows_make_pixels_irrelevant(orc, small):
    cat = dict(small)
    row = small["los"][0]
    cat["los"] = np.stack([row, row, row])
    a = orc.loglik(cat, FIDUCIAL, neff_min_event=0.0)
    cat2 = dict(cat)
    cat2["pix"] = np.random.default_rng(3).integers(0, 3, size=len(cat["pix"])).astype(np.int32)
    b = orc.loglik(cat2, FIDUCIAL, neff_min_event=0.0)
    np.testing.assert_array_equal(a["lnL_event"], b["lnL_event"])
    assert a["lnL_total"][0] == b["lnL_total"][0]


def test_h0_distance_scaling(orc, small):
    # d_L -> 2 d_L (exact in float32) with H0 -> H0 / 2 leaves x = d_L H0 / c, hence z,
    # unchanged; every ln w shifts by -ln 2 (the d d_L / dz Jacobian), so each ln L_i and
    # ln xi shift by -ln 2 and the total is unchanged.
    cat = dict(small)
    cat["dl"] = small["dl"] * np.float32(2.0)
    cat["inj_dl"] = small["inj_dl"] * np.float32(2.0)
    lam2 = FIDUCIAL.copy()
    lam2[0] /= 2.0
    a = orc.loglik(small, FIDUCIAL, neff_min_event=0.0)
    b = orc.loglik(cat, lam2, neff_min_event=0.0)
    np.testing.assert_allclose(b["lnL_event"] - a["lnL_event"], -math.log(2.0), atol=1e-11)
    assert b["ln_xi"][0] - a["ln_xi"][0] == pytest.approx(-math.log(2.0), abs=1e-11)
    assert b["lnL_total"][0] == pytest.approx(a["lnL_total"][0], abs=1e-9)


def test_selection_identity(orc, cat_c1):
    # when ln p_draw is the population's own detector-frame density at Lambda0, every
    # ratio is one: xi(Lambda0) = N_found / N_draw and N_eff,sel = N_found exactly
    row = smooth_row(257)
    m1, m2, dl = cat_c1["inj_m1"][:400], cat_c1["inj_m2"][:400], cat_c1["inj_dl"][:400]
    lp = orc.ln_w_row(FIDUCIAL, m1, m2, dl, np.zeros(400, np.float32), row, 2.0)
    ok = np.isfinite(lp)
    assert ok.sum() > 100
    # store the density as float32 and compare in the same precision it was stored in
    lpd = lp[ok].astype(np.float32)
    inj = list(zip(m1[ok], m2[ok], dl[ok], lpd))
    ev = [[(cat_c1["m1"][0], cat_c1["m2"][0], cat_c1["dl"][0], cat_c1["lnpe"][0], 0)]]
    cat = tiny_catalogue([row, row], ev, inj, n_draw=5000.0)
    out = orc.loglik(cat, FIDUCIAL, neff_min_event=0.0)
    n = int(ok.sum())
    resid = lp[ok] - lpd.astype(np.float64)    # float32 storage error of each ratio
    expect = math.log(np.sum(np.exp(resid))) - math.log(5000.0)
    assert out["ln_xi"][0] == pytest.approx(expect, abs=1e-12)
    assert out["ln_xi"][0] == pytest.approx(math.log(n / 5000.0), abs=1e-6)
    assert out["neff_sel"][0] == pytest.approx(n, rel=1e-9)


def test_detector_frame_density_integrates_to_one(orc):
    # exp(ln w) with pi_PE = 1 is the population density in (m1_det, m2_det, d_L);
    # integrating it over detector-frame space (own Gauss-Legendre product rule, no
    # change of variables) must give 1, which fixes the (1+z)^2 mass Jacobian, the
    # d d_L/dz Jacobian, the 1/(1+z) time dilation and every normaliser at once.
    lam = FIDUCIAL.copy()
    lam[0], lam[1] = 68.0, 0.31
    zmax = 2.0
    row = smooth_row(2049, zmax)
    H0, om = lam[0], lam[1]
    dlmax = C_KMS / H0 * orc.D(zmax, om)
    xg, wg = np.polynomial.legendre.leggauss(16)

    def gl(a, b):
        return 0.5 * (b - a) * xg + 0.5 * (a + b), 0.5 * (b - a) * wg

    dl_nodes, dl_w = [], []
    edges = np.linspace(0.0, dlmax, 9)
    for a, b in zip(edges[:-1], edges[1:]):
        x, w = gl(a, b)
        dl_nodes.append(x)
        dl_w.append(w)
    dl_nodes, dl_w = np.concatenate(dl_nodes), np.concatenate(dl_w)
    pts, wts = [], []
    mmin, mmax, dm, mu, sig = lam[4], lam[5], lam[6], lam[7], lam[8]
    for d, wd in zip(dl_nodes, dl_w):
        z = orc.z_of_x(d * H0 / C_KMS, om, zmax)
        u = 1.0 + z
        cuts1 = [mmin * u, (mmin + dm) * u, (mu - 4 * sig) * u, (mu + 4 * sig) * u, mmax * u]
        for a, b in zip(cuts1[:-1], cuts1[1:]):
            x1, w1 = gl(a, b)
            for m1, v1 in zip(x1, w1):
                cuts2 = [mmin * u] + [c for c in ((mmin + dm) * u,) if c < m1] + [m1]
                for a2, b2 in zip(cuts2[:-1], cuts2[1:]):
                    x2, w2 = gl(a2, b2)
                    pts.append(np.stack([np.full(16, m1), x2, np.full(16, d)], axis=1))
                    wts.append(w2 * v1 * wd)
    pts, wts = np.concatenate(pts), np.concatenate(wts)
    lw = orc.ln_w_row(lam, pts[:, 0], pts[:, 1], pts[:, 2], np.zeros(len(pts)), row, zmax)
    # the sample points are rounded to float32; integrate with the same rounded points
    tot = np.sum(np.where(np.isfinite(lw), np.exp(lw), 0.0) * wts)
    assert tot == pytest.approx(1.0, abs=1e-6)


def test_flags(orc, small):
    bad = FIDUCIAL.copy()
    bad[5] = 4.0  # m_max below m_min
    out = orc.loglik(small, np.stack([FIDUCIAL, bad]), neff_min_event=0.0)
    assert out["flags"][0] == 0 and np.isfinite(out["lnL_total"][0])
    assert out["flags"][1] == 1 and out["lnL_total"][1] == -math.inf
    assert np.all(out["lnL_event"][1] == -math.inf)
    out = orc.loglik(small, FIDUCIAL, neff_min_event=1e9)
    assert out["flags"][0] & 2 and out["lnL_total"][0] == -math.inf
    out = orc.loglik(small, FIDUCIAL, neff_min_event=0.0, neff_min_sel=1e9)
    assert out["flags"][0] & 4 and out["lnL_total"][0] == -math.inf
    # an event whose samples all lie beyond z_max has no weight
    cat = dict(small)
    cat["dl"] = small["dl"].copy()
    cat["dl"][: small["offsets"][1]] = np.float32(1e6)
    out = orc.loglik(cat, FIDUCIAL, neff_min_event=2.0)
    assert out["lnL_event"][0, 0] == -math.inf and out["neff_event"][0, 0] == 0.0
    assert out["flags"][0] & 2


def test_invalid_inputs_rejected(orc, small):
    cat = dict(small)
    cat["pix"] = small["pix"].copy()
    cat["pix"][0] = 3
    with pytest.raises(ValueError):
        orc.loglik(cat, FIDUCIAL)
    cat = dict(small)
    cat["offsets"] = small["offsets"].copy()
    cat["offsets"][2] = cat["offsets"][1]
    with pytest.raises(ValueError):
        orc.loglik(cat, FIDUCIAL)


def test_gradient_matches_finite_differences(orc, small):
    # central differences with small steps: the piecewise-linear LOS interpolation has
    # kinks at grid nodes, so the derivative is the cell-local (a.e.) one and a large
    # step would straddle kinks
    lam = FIDUCIAL.copy()
    g = orc.loglik(small, lam, grad=True, neff_min_event=0.0)["grad_total"][0]
    scale = np.maximum(np.abs(lam), 0.1)
    for i in range(13):
        h = 1e-6 * scale[i]
        lp, lm = lam.copy(), lam.copy()
        lp[i] += h
        lm[i] -= h
        fp = orc.loglik(small, lp, neff_min_event=0.0)["lnL_total"][0]
        fm = orc.loglik(small, lm, neff_min_event=0.0)["lnL_total"][0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 2e-7 / scale[i], (i, fd, g[i])
