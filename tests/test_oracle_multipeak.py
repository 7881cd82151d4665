"""Pins of the oracle's multi-peak mass model (the model of the paper's simulated O5
catalogue, App. A, Table 2): a power law and two truncated Gaussian peaks, mixed as
(1 - lam_g) P + lam_g [lam_low G_low + (1 - lam_low) G_high], smoothed and normalised
like the single-peak model.

What fixes it independently of the oracle's formulas: at lam_low = 1 (or 0) it is the
already-pinned power law + peak model with the low (or high) Gaussian; exchanging the
two Gaussians together with lam_low <-> 1 - lam_low changes nothing; without smoothing
(delta_m = 0) the density is the textbook mixture of a normalised power law and two
scipy truncated normals; the density integrates to one under an independent
quadrature; the 16-component gradient matches central finite differences inside the
domain and one-sided differences (taken into the domain) at the mixture weights' bounds.
"""
import os

import numpy as np
import pytest

from conftest import smooth_row, tiny_catalogue
from paper_2605_23538_gb300.synth import FIDUCIAL_MP, LAMBDA_NAMES_MP

P_MU, P_SIG, P_LAM, P_MU2, P_SIG2, P_LAM1 = 7, 8, 9, 13, 14, 15
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_multipeak.txt")


def _with(lam, **kw):
    out = np.array(lam, dtype=np.float64)
    for k, v in kw.items():
        out[LAMBDA_NAMES_MP.index(k)] = v
    return out


def _swapped(lam):
    """The same population with the two Gaussians exchanged."""
    s = np.array(lam, dtype=np.float64)
    s[[P_MU, P_SIG, P_MU2, P_SIG2]] = lam[[P_MU2, P_SIG2, P_MU, P_SIG]]
    s[P_LAM1] = 1.0 - lam[P_LAM1]
    return s


@pytest.fixture(scope="module")
def small(cat_c1):
    rng = np.random.default_rng(15)
    row = smooth_row(257)
    rows = np.stack([row, row * np.float32(1.4), row * np.float32(0.6)])
    idx = rng.integers(0, len(cat_c1["m1"]), size=(4, 40))
    ev = [[(cat_c1["m1"][k], cat_c1["m2"][k], cat_c1["dl"][k], cat_c1["lnpe"][k], int(rng.integers(0, 3)))
           for k in idx[e]] for e in range(4)]
    ki = rng.integers(0, len(cat_c1["inj_m1"]), size=300)
    inj = [(cat_c1["inj_m1"][i], cat_c1["inj_m2"][i], cat_c1["inj_dl"][i], cat_c1["inj_lnpd"][i]) for i in ki]
    return tiny_catalogue(rows, ev, inj, n_draw=1000.0)


def test_table2_point_is_the_papers():
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    names = tuple(r[0] for r in rows)
    vals = np.array([float(r[1]) for r in rows])
    assert names == LAMBDA_NAMES_MP
    np.testing.assert_array_equal(vals, FIDUCIAL_MP)


@pytest.mark.parametrize("lam_low", [1.0, 0.0])
def test_reduces_to_power_law_plus_peak(orc, small, lam_low):
    mp = _with(FIDUCIAL_MP, lambda_low=lam_low)
    plp = mp[:13].copy()
    if lam_low == 0.0:                       # the high-mass Gaussian is the only peak
        plp[P_MU], plp[P_SIG] = mp[P_MU2], mp[P_SIG2]
    for m in np.linspace(4.0, 90.0, 173):
        a, b = orc.ln_p_m1(m, mp), orc.ln_p_m1(m, plp)
        assert (a == b == -np.inf) or a == pytest.approx(b, abs=1e-12)
        assert orc.ln_p_m2(0.7 * m, m, mp) == orc.ln_p_m2(0.7 * m, m, plp)
    assert orc.ln_Zm1(mp) == pytest.approx(orc.ln_Zm1(plp), abs=1e-13)
    r_mp = orc.loglik(small, mp, grad=True, neff_min_event=0.0)
    r_pl = orc.loglik(small, plp, grad=True, neff_min_event=0.0)
    np.testing.assert_allclose(r_mp["lnL_event"], r_pl["lnL_event"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(r_mp["ln_xi"], r_pl["ln_xi"], rtol=0, atol=1e-10)
    g_mp, g_pl = r_mp["grad_total"][0], r_pl["grad_total"][0]
    assert g_mp.shape == (16,)
    # the remaining Gaussian's parameters sit in slots 7, 8 (lam_low = 1) or 13, 14 (0)
    keep = list(range(13)) if lam_low == 1.0 else [i for i in range(13) if i not in (P_MU, P_SIG)]
    np.testing.assert_allclose(g_mp[keep], g_pl[keep], rtol=1e-9, atol=1e-9)
    if lam_low == 1.0:
        assert g_mp[P_MU2] == 0.0 and g_mp[P_SIG2] == 0.0
    else:
        np.testing.assert_allclose(g_mp[[P_MU2, P_SIG2]], g_pl[[P_MU, P_SIG]], rtol=1e-9, atol=1e-9)
        assert g_mp[P_MU] == 0.0 and g_mp[P_SIG] == 0.0


def test_exchanging_the_peaks_is_a_symmetry(orc, small):
    lam = FIDUCIAL_MP
    sw = _swapped(lam)
    for m in np.linspace(4.0, 90.0, 97):
        a, b = orc.ln_p_m1(m, lam), orc.ln_p_m1(m, sw)
        assert (a == b == -np.inf) or a == pytest.approx(b, abs=1e-12)
    r = orc.loglik(small, lam, grad=True, neff_min_event=0.0)
    s = orc.loglik(small, sw, grad=True, neff_min_event=0.0)
    np.testing.assert_allclose(s["lnL_total"], r["lnL_total"], rtol=0, atol=1e-9)
    g, h = r["grad_total"][0], s["grad_total"][0]
    perm = np.arange(16)
    perm[[P_MU, P_SIG, P_MU2, P_SIG2]] = [P_MU2, P_SIG2, P_MU, P_SIG]
    want = g[perm]
    want[P_LAM1] = -g[P_LAM1]
    np.testing.assert_allclose(h, want, rtol=1e-8, atol=1e-8)


def test_hard_cut_density_is_the_textbook_mixture(orc):
    stats = pytest.importorskip("scipy.stats")
    lam = _with(FIDUCIAL_MP, delta_m=0.0)
    a, mmin, mmax = lam[2], lam[4], lam[5]
    lg, ll = lam[P_LAM], lam[P_LAM1]

    def tn(m, mu, sig):
        return stats.truncnorm.pdf(m, (mmin - mu) / sig, (mmax - mu) / sig, loc=mu, scale=sig)

    for m in np.linspace(mmin + 1e-6, mmax - 1e-6, 211):
        pl = (1.0 - a) * m ** -a / (mmax ** (1.0 - a) - mmin ** (1.0 - a))
        want = (1.0 - lg) * pl + lg * (ll * tn(m, lam[P_MU], lam[P_SIG]) + (1.0 - ll) * tn(m, lam[P_MU2], lam[P_SIG2]))
        assert orc.ln_p_m1(m, lam) == pytest.approx(np.log(want), abs=1e-10)
    assert orc.ln_p_m1(mmax + 0.1, lam) == -np.inf and orc.ln_p_m1(mmin - 0.1, lam) == -np.inf


@pytest.mark.parametrize("lam", [FIDUCIAL_MP, _with(FIDUCIAL_MP, lambda_g=0.9, lambda_low=0.3, sigma_low=2.0)])
def test_primary_mass_density_integrates_to_one(orc, lam):
    integrate = pytest.importorskip("scipy.integrate")
    mmin, mmax, dm = lam[4], lam[5], lam[6]
    f = lambda m: np.exp(orc.ln_p_m1(m, lam))
    pts = sorted(p for p in (mmin + dm, lam[P_MU], lam[P_MU2]) if mmin < p < mmax)
    edges = [mmin] + pts + [mmax]
    total = sum(integrate.quad(f, lo, hi, epsabs=1e-13, epsrel=1e-12, limit=400)[0]
                for lo, hi in zip(edges[:-1], edges[1:]))
    assert total == pytest.approx(1.0, abs=1e-9)


def test_gradient_matches_finite_differences(orc, small):
    lam = FIDUCIAL_MP.copy()
    g = orc.loglik(small, lam, grad=True, neff_min_event=0.0)["grad_total"][0]
    scale = np.maximum(np.abs(lam), 0.1)
    for i in range(16):
        h = 1e-6 * scale[i]
        lp, lm = lam.copy(), lam.copy()
        lp[i] += h
        lm[i] -= h
        fp = orc.loglik(small, lp, neff_min_event=0.0)["lnL_total"][0]
        fm = orc.loglik(small, lm, neff_min_event=0.0)["lnL_total"][0]
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 2e-7 / scale[i], (LAMBDA_NAMES_MP[i], fd, g[i])
    # the three new parameters do move the likelihood at this point
    assert np.all(np.abs(g[[P_MU2, P_SIG2, P_LAM1]]) > 1e-3)


@pytest.mark.parametrize("bound", [(1.0, None), (0.0, None), (None, 1.0), (None, 0.0), (1.0, 0.0), (0.0, 1.0)])
def test_gradient_at_the_mixture_bounds_is_one_sided(orc, small, bound):
    # at lambda_g or lambda_low = 0 or 1 only one side of the point is in the domain: the
    # oracle's derivative of those two components must equal the one-sided difference
    # taken into the domain (second order: three points)
    lam = FIDUCIAL_MP.copy()
    if bound[0] is not None:
        lam[P_LAM] = bound[0]
    if bound[1] is not None:
        lam[P_LAM1] = bound[1]
    g = orc.loglik(small, lam, grad=True, neff_min_event=0.0)["grad_total"][0]
    assert np.all(np.isfinite(g))
    f0 = orc.loglik(small, lam, neff_min_event=0.0)["lnL_total"][0]
    for i in (P_LAM, P_LAM1):
        d = -1.0 if lam[i] >= 1.0 else 1.0             # the direction into the domain
        h = 1e-5
        l1, l2 = lam.copy(), lam.copy()
        l1[i] += d * h
        l2[i] += 2 * d * h
        f1 = orc.loglik(small, l1, neff_min_event=0.0)["lnL_total"][0]
        f2 = orc.loglik(small, l2, neff_min_event=0.0)["lnL_total"][0]
        fd = d * (-3.0 * f0 + 4.0 * f1 - f2) / (2.0 * h)
        assert abs(fd - g[i]) <= 1e-5 * abs(g[i]) + 1e-5, (bound, LAMBDA_NAMES_MP[i], fd, g[i])
    if lam[P_LAM] == 0.0:                              # no lambda_low dependence without the peaks
        assert g[P_LAM1] == 0.0


@pytest.mark.parametrize("bad", [dict(sigma_high=0.0), dict(sigma_high=-1.0), dict(lambda_low=1.01),
                                 dict(lambda_low=-0.01), dict(mu_high=np.nan)])
def test_outside_the_domain_is_flagged(orc, small, bad):
    r = orc.loglik(small, _with(FIDUCIAL_MP, **bad))
    assert r["flags"][0] == 1 and r["lnL_total"][0] == -np.inf


def test_rows_of_other_widths_are_rejected(orc, small):
    with pytest.raises(AssertionError):
        orc.loglik(small, FIDUCIAL_MP[:14])
