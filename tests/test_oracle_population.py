"""Pins for the oracle's population model (power law + peak masses, Madau-Dickinson rate).

The paper names these models without writing them; the pins check the literature
definitions through properties they must have: textbook normalisations when the
smoothing and the peak are switched off (and the alpha = 1, beta = -1 logarithmic
limits), unit normalisation of p(m1) and of p(m2 | m1) by an independent quadrature,
the symmetry of the smoothing window, the truncated normal at lambda = 1, and the
rate's psi(0) = 1, peak location and asymptotic slopes.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from paper_2605_23538_gb300.synth import FIDUCIAL

H0, OM, ALPHA, BETA, MMIN, MMAX, DM, MU, SIG, LAM, GAM, KAP, ZP = range(13)


def lam_with(**kw):
    lam = FIDUCIAL.copy()
    names = dict(alpha=ALPHA, beta=BETA, mmin=MMIN, mmax=MMAX, dm=DM, mu=MU, sig=SIG, lam=LAM,
                 gam=GAM, kap=KAP, zp=ZP)
    for k, v in kw.items():
        lam[names[k]] = v
    return lam


@pytest.mark.parametrize("alpha", [3.4, 2.2, 0.5])
@pytest.mark.parametrize("m1", [5.5, 17.0, 89.0])
def test_power_law_textbook(orc, alpha, m1):
    lam = lam_with(alpha=alpha, dm=0.0, lam=0.0)
    a = 1.0 - alpha
    ref = math.log(a / (90.0 ** a - 5.0 ** a)) - alpha * math.log(m1)
    assert orc.ln_p_m1(m1, lam) == pytest.approx(ref, abs=1e-12)


def test_power_law_alpha_one_log_limit(orc):
    lam = lam_with(alpha=1.0, dm=0.0, lam=0.0)
    for m1 in (5.5, 30.0, 89.0):
        ref = -math.log(m1) - math.log(math.log(90.0 / 5.0))
        assert orc.ln_p_m1(m1, lam) == pytest.approx(ref, abs=1e-12)


@pytest.mark.parametrize("beta", [1.1, -0.5, 3.0])
@pytest.mark.parametrize("m1,m2", [(30.0, 12.0), (80.0, 79.0), (9.0, 5.2)])
def test_pairing_textbook(orc, beta, m1, m2):
    lam = lam_with(beta=beta, dm=0.0)
    b = 1.0 + beta
    ref = math.log(b / (m1 ** b - 5.0 ** b)) + beta * math.log(m2)
    assert orc.ln_p_m2(m2, m1, lam) == pytest.approx(ref, abs=1e-12)


def test_pairing_beta_minus_one_log_limit(orc):
    lam = lam_with(beta=-1.0, dm=0.0)
    for m1, m2 in ((30.0, 12.0), (80.0, 6.0)):
        ref = -math.log(m2) - math.log(math.log(m1 / 5.0))
        assert orc.ln_p_m2(m2, m1, lam) == pytest.approx(ref, abs=1e-12)


def test_peak_only_is_truncated_normal(orc):
    lam = lam_with(lam=1.0, dm=0.0, mu=34.0, sig=4.0)
    a, b = (5.0 - 34.0) / 4.0, (90.0 - 34.0) / 4.0
    for m1 in (6.0, 25.0, 34.0, 41.0, 60.0):
        ref = stats.truncnorm.logpdf(m1, a, b, loc=34.0, scale=4.0)
        assert orc.ln_p_m1(m1, lam) == pytest.approx(ref, abs=1e-10)


def test_smoothing_window_values(orc):
    mmin, dm = 5.0, 4.0
    assert orc.S(mmin, mmin, dm) == 0.0
    assert orc.S(mmin - 1e-9, mmin, dm) == 0.0
    assert orc.S(mmin + dm, mmin, dm) == 1.0
    assert orc.S(mmin + 0.5 * dm, mmin, dm) == pytest.approx(0.5, abs=1e-15)
    xs = np.linspace(1e-3, dm - 1e-3, 37)
    s = np.array([orc.S(mmin + x, mmin, dm) for x in xs])
    assert np.all(np.diff(s) > 0)
    # f(m') = dm/m' + dm/(m' - dm) is odd about dm/2, so S(a) + S(dm - a) = 1
    for x in xs:
        assert orc.S(mmin + x, mmin, dm) + orc.S(mmin + dm - x, mmin, dm) == pytest.approx(1.0, abs=1e-14)
    # delta_m = 0: a hard step at m_min
    assert orc.S(mmin, mmin, 0.0) == 1.0
    assert orc.S(mmin - 1e-12, mmin, 0.0) == 0.0


@pytest.mark.parametrize("lam", [FIDUCIAL, lam_with(lam=0.3, dm=6.0, alpha=2.0, sig=7.0)])
def test_primary_mass_unit_normalisation(orc, lam):
    f = lambda m: math.exp(orc.ln_p_m1(m, lam))
    mw = lam[MMIN] + lam[DM]
    pts = [mw, lam[MU] - 3 * lam[SIG], lam[MU], lam[MU] + 3 * lam[SIG]]
    tot = integrate.quad(f, lam[MMIN], lam[MMAX], points=pts, epsabs=0, epsrel=1e-12, limit=400)[0]
    assert tot == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("m1", [6.0, 8.5, 9.0, 30.0, 89.0])
def test_pairing_unit_normalisation(orc, m1):
    lam = FIDUCIAL
    f = lambda m: math.exp(orc.ln_p_m2(m, m1, lam))
    pts = [p for p in (lam[MMIN] + lam[DM],) if p < m1]
    tot = integrate.quad(f, lam[MMIN], m1, points=pts or None, epsabs=0, epsrel=1e-12, limit=400)[0]
    assert tot == pytest.approx(1.0, abs=1e-9)


def test_mass_support(orc):
    lam = FIDUCIAL
    assert orc.ln_p_m1(90.0001, lam) == -math.inf
    assert orc.ln_p_m1(4.99, lam) == -math.inf
    assert orc.ln_p_m2(31.0, 30.0, lam) == -math.inf
    assert orc.ln_p_m2(4.99, 30.0, lam) == -math.inf


@pytest.mark.parametrize("g,k,zp", [(2.7, 3.0, 2.0), (3.3, 2.9, 2.5), (1.0, 5.0, 0.5)])
def test_rate_unity_at_zero_and_peak(orc, g, k, zp):
    lam = lam_with(gam=g, kap=k, zp=zp)
    assert orc.ln_psi(0.0, lam) == pytest.approx(0.0, abs=1e-15)
    # d ln psi / dz = 0 at (1 + z*) = (1 + zp) (g / k)^(1 / (g + k))
    zs = (1.0 + zp) * (g / k) ** (1.0 / (g + k)) - 1.0
    if zs > 1e-3:
        h = 1e-4
        d = (orc.ln_psi(zs + h, lam) - orc.ln_psi(zs - h, lam)) / (2 * h)
        assert abs(d) < 1e-7
        assert orc.ln_psi(zs, lam) > orc.ln_psi(zs + 0.05, lam)
        assert orc.ln_psi(zs, lam) > orc.ln_psi(zs - 0.05, lam)


def test_rate_asymptotic_slopes(orc):
    # far below the peak psi -> (1+z)^gamma; far above it psi -> (1+z)^-kappa
    lo = lam_with(gam=2.7, kap=3.0, zp=1e5)
    hi = lam_with(gam=2.7, kap=3.0, zp=-1.0 + 1e-6)
    for z in (0.3, 1.0, 2.0):
        assert orc.ln_psi(z, lo) == pytest.approx(2.7 * math.log1p(z), abs=1e-9)
        assert orc.ln_psi(z, hi) == pytest.approx(-3.0 * math.log1p(z), abs=1e-9)
    flat = lam_with(gam=0.0, kap=0.0)
    for z in (0.0, 0.7, 2.0):
        assert orc.ln_psi(z, flat) == pytest.approx(0.0, abs=1e-15)


def test_redshift_normalisation(orc):
    # flat rate (gamma = kappa = 0, psi = 1) and a constant LOS row: N_z is the
    # trapezoid sum of 1/(1+z), which tends to ln 3 on [0, 2] as the grid refines.
    lam = lam_with(gam=0.0, kap=0.0)
    for n in (5, 513):
        z = np.linspace(0.0, 2.0, n)
        w = np.full(n, z[1])
        w[0] = w[-1] = 0.5 * z[1]
        ref = float(np.sum(w * 0.5 / (1 + z)))
        assert orc.ln_Nz(lam, np.full(n, 0.5), 2.0) == pytest.approx(math.log(ref), abs=1e-14)
    assert orc.ln_Nz(lam, np.ones(8193), 2.0) == pytest.approx(math.log(math.log(3.0)), abs=1e-8)
