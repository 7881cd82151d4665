"""Brute force: a separate high-precision restatement of the estimator on tiny inputs.

Everything is re-derived here with mpmath at 30 significant digits, directly from the
definitions (Eq. 1 for d_L, Eqs. 2-7 for the likelihood with the zero-width kernel):
tanh-sinh quadrature instead of Gauss-Kronrod, bisection instead of Newton, explicit
sums instead of logsumexp.  It shares no code with the oracle.  2 events x 3 samples,
4 injections, 3 pixels x 5 redshift nodes, with samples placed inside and outside
the smoothing window and one sample beyond z_max.
"""
import math
import os

import numpy as np
import pytest

from conftest import tiny_catalogue

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30

C = mp.mpf("299792.458")


def _table2():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_injected_hyperparameters.txt")
    vals = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [float(v) for _, v in vals]


LAM = _table2()   # App. A, Table 2
ROWS = [[0.10, 0.80, 0.55, 0.30, 0.20],
        [0.30, 0.40, 0.70, 0.25, 0.10],
        [0.05, 0.60, 0.60, 0.45, 0.05]]
ZMAX = 2.0
EVENTS = [
    [(45.0, 30.0, 2500.0, 15.7, 0), (11.0, 9.0, 1800.0, 15.0, 1), (60.0, 55.0, 4000.0, 16.6, 2)],
    [(20.0, 12.0, 900.0, 13.6, 2), (35.0, 34.0, 6500.0, 17.5, 0), (70.0, 20.0, 1e5, 23.0, 1)],
]
INJ = [(50.0, 40.0, 3000.0, -18.0), (12.0, 7.5, 1500.0, -15.5), (90.0, 10.0, 5000.0, -20.0),
       (25.0, 24.0, 800.0, -14.0)]
N_DRAW = 37.0


def f32(x):
    return mp.mpf(float(np.float32(x)))


def E(z, om):
    return mp.sqrt(om * (1 + z) ** 3 + 1 - om)


def I(z, om):
    return mp.quad(lambda t: 1 / E(t, om), [0, z])


def D(z, om):
    return (1 + z) * I(z, om)


def z_of(x, om):
    lo, hi = mp.mpf(0), mp.mpf(ZMAX)
    for _ in range(110):
        mid = (lo + hi) / 2
        if D(mid, om) > x:
            hi = mid
        else:
            lo = mid
    return (lo + hi) / 2


def S(m, mmin, dm):
    if m < mmin:
        return mp.mpf(0)
    if m >= mmin + dm:
        return mp.mpf(1)
    mp_ = m - mmin
    if mp_ == 0:
        return mp.mpf(0)
    return 1 / (1 + mp.exp(dm / mp_ + dm / (mp_ - dm)))


def population(lam):
    H0, om, a, b, mmin, mmax, dm, mu, sg, lp, g, k, zp = [mp.mpf(v) for v in lam]
    ZP = mp.quad(lambda m: m ** -a, [mmin, mmax])
    ZG = mp.quad(lambda m: mp.npdf(m, mu, sg), [mmin, mu, mmax])

    def mix(m):
        return (1 - lp) * m ** -a / ZP + lp * mp.npdf(m, mu, sg) / ZG

    Zm1 = mp.quad(lambda m: mix(m) * S(m, mmin, dm), [mmin, mmin + dm, mu, mmax])

    def p1(m):
        if m > mmax or m < mmin:
            return mp.mpf(0)
        return mix(m) * S(m, mmin, dm) / Zm1

    def p2(m2, m1):
        if m2 > m1 or m2 < mmin:
            return mp.mpf(0)
        pts = [mmin] + ([mmin + dm] if mmin + dm < m1 else []) + [m1]
        Cm = mp.quad(lambda m: m ** b * S(m, mmin, dm), pts)
        return m2 ** b * S(m2, mmin, dm) / Cm

    def psi(z):
        return (1 + (1 + zp) ** (-g - k)) * (1 + z) ** g / (1 + ((1 + z) / (1 + zp)) ** (g + k))

    return H0, om, p1, p2, psi


def lerp(row, z):
    if z < 0 or z > ZMAX:
        return mp.mpf(0)
    n = len(row)
    pos = z * (n - 1) / ZMAX
    j = min(int(mp.floor(pos)), n - 2)
    t = pos - j
    return row[j] * (1 - t) + row[j + 1] * t


def weight(lam, pop, row, Nz, m1d, m2d, dl, lnpi):
    H0, om, p1, p2, psi = pop
    m1d, m2d, dl, lnpi = f32(m1d), f32(m2d), f32(dl), f32(lnpi)
    x = dl * H0 / C
    if x > D(mp.mpf(ZMAX), om):
        return mp.mpf(0)
    z = z_of(x, om)
    u = 1 + z
    m1, m2 = m1d / u, m2d / u
    pz = lerp(row, z) * psi(z) / u / Nz
    pm = p1(m1) * p2(m2, m1)
    ddl = (C / H0) * (I(z, om) + u / E(z, om))
    return pz * pm / (u * u * ddl) / mp.exp(lnpi)


def brute(lam):
    pop = population(lam)
    rows = [[f32(v) for v in r] for r in ROWS]          # the LOS table is float32 input
    pbar = [sum(r[j] for r in rows) / len(rows) for j in range(len(rows[0]))]
    dz = mp.mpf(ZMAX) / (len(pbar) - 1)
    Nz = sum((mp.mpf("0.5") if j in (0, len(pbar) - 1) else 1) * pbar[j] * pop[4](j * dz) / (1 + j * dz)
             for j in range(len(pbar))) * dz
    lnL = []
    for ev in EVENTS:
        w = [weight(lam, pop, rows[s[4]], Nz, *s[:4]) for s in ev]
        lnL.append(mp.log(sum(w) / len(w)))
    ws = [weight(lam, pop, pbar, Nz, *s) for s in INJ]
    ln_xi = mp.log(sum(ws) / N_DRAW)
    return lnL, ln_xi, sum(lnL) - len(EVENTS) * ln_xi


@pytest.fixture(scope="module")
def tiny():
    return tiny_catalogue(ROWS, EVENTS, INJ, N_DRAW, ZMAX)


@pytest.mark.parametrize("lam", [LAM, [70.0, 0.3, 3.4, 1.1, 5.0, 90.0, 4.0, 34.0, 4.0, 0.04, 2.7, 3.0, 2.0]])
def test_oracle_matches_brute_force(orc, tiny, lam):
    lnL, ln_xi, total = brute(lam)
    out = orc.loglik(tiny, np.array(lam), neff_min_event=0.0)
    assert out["flags"][0] == 0
    for e in range(len(EVENTS)):
        assert out["lnL_event"][0, e] == pytest.approx(float(lnL[e]), abs=1e-11)
    assert out["ln_xi"][0] == pytest.approx(float(ln_xi), abs=1e-11)
    assert out["lnL_total"][0] == pytest.approx(float(total), abs=1e-10)


def test_the_tiny_case_exercises_every_branch(orc, tiny):
    lam = np.array(LAM)
    lw = [orc.ln_w_row(lam, [s[0]], [s[1]], [s[2]], [s[3]], np.array(ROWS[s[4]], np.float32), ZMAX)[0]
          for ev in EVENTS for s in ev]
    assert sum(1 for v in lw if v == -math.inf) >= 1          # a sample beyond z_max
    # and a sample whose source-frame masses sit inside the smoothing window
    x = 1800.0 * 67.4 / 299792.458
    z = orc.z_of_x(x, 0.315, ZMAX)
    assert 4.6 < 9.0 / (1 + z) < 4.6 + 4.8
