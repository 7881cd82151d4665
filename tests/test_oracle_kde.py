"""Pins of the oracle's KDE form of the likelihood (Eqs. 5-7) and its bandwidth rules.

The anchor is the kernel's zero-width limit: when every pixel's LOS prior is linear in z
and all samples sit well inside the redshift grid, Gaussian smoothing leaves a linear
function unchanged and the trapezoid rule integrates it exactly, so the KDE event term
must equal the (already pinned) Monte-Carlo event term for any bandwidth.  A mistake in
the kernel's normalisation, the grid, the trapezoid weights, the weight w' or the LOS
product breaks that equality.  The bandwidth rules are checked against numpy's standard
deviation and percentiles, scale equivariance, and the biweight's resistance to outliers.
"""
import numpy as np
import pytest

from conftest import tiny_catalogue


def test_scott_and_silverman_match_numpy(orc):
    r = np.random.default_rng(7)
    for n in (2, 3, 10, 257, 4000):
        z = r.gamma(3.0, 0.1, size=n)
        sd = np.std(z, ddof=1)
        assert orc.bandwidth(z, "scott") == pytest.approx(1.06 * sd * n ** -0.2, rel=1e-12)
        iqr = np.percentile(z, 75) - np.percentile(z, 25)
        assert orc.bandwidth(z, "silverman") == pytest.approx(0.9 * min(sd, iqr / 1.34) * n ** -0.2, rel=1e-12)


def test_bandwidths_are_scale_equivariant(orc):
    z = np.random.default_rng(8).normal(0.7, 0.05, 500)
    for rule in ("scott", "silverman", "biweight"):
        h = orc.bandwidth(z, rule)
        assert h > 0
        assert orc.bandwidth(3.5 * z - 2.0, rule) == pytest.approx(3.5 * h, rel=1e-10)
        assert orc.bandwidth(-z, rule) == pytest.approx(h, rel=1e-10)


def test_biweight_scale_of_a_gaussian_and_outlier_resistance(orc):
    r = np.random.default_rng(9)
    sigma, n = 0.08, 200_000
    z = r.normal(1.0, sigma, n)
    s_bi = orc.bandwidth(z, "biweight") / (1.06 * n ** -0.2)
    assert s_bi == pytest.approx(sigma, rel=0.02)        # the midvariance of a normal is ~sigma^2
    small = r.normal(1.0, sigma, 400)
    spoiled = np.concatenate([small, [40.0, 55.0, -30.0]])  # far beyond 9 MAD
    shrink = (403 / 400) ** -0.2
    assert orc.bandwidth(spoiled, "biweight") == pytest.approx(orc.bandwidth(small, "biweight") * shrink, rel=0.05)
    assert orc.bandwidth(spoiled, "scott") > 30 * orc.bandwidth(small, "scott")


def test_degenerate_pixels_have_no_bandwidth(orc):
    assert orc.bandwidth(np.array([0.4]), "scott") == 0.0
    assert orc.bandwidth(np.full(5, 0.4), "biweight") == 0.0


def _linear_los_catalogue(synth, seed=3, n_pix=3, per_pix=(40, 60, 25), z_max=2.0, n_z=400):
    """Three pixels with LOS priors linear in z and samples at z ~ 0.5-0.9."""
    r = np.random.default_rng(seed)
    zg = np.linspace(0.0, z_max, n_z)
    rows = []
    for j in range(n_pix):
        a, b = 0.2 + 0.1 * j, 0.4 - 0.15 * j
        row = a + b * zg
        rows.append(row / (z_max * (a + 0.5 * b * z_max)))
    events = []
    for e in range(2):
        ev = []
        for j in range(n_pix):
            for _ in range(per_pix[j]):
                dl = r.uniform(3000.0, 6000.0)
                m1 = r.uniform(25.0, 60.0)
                m2 = m1 * r.uniform(0.4, 0.95)
                ev.append((m1, m2, dl, 2.0 * np.log(dl), j))
        events.append(ev)
    inj = []
    for _ in range(400):
        dl = r.uniform(500.0, 9000.0)
        m1 = np.exp(r.uniform(np.log(8.0), np.log(150.0)))
        m2 = m1 * r.uniform(0.2, 1.0)
        inj.append((m1, m2, dl, -18.0))
    return tiny_catalogue(np.array(rows, np.float32), events, inj, 4000.0, z_max)


@pytest.mark.parametrize("rule", ["scott", "silverman", "biweight"])
@pytest.mark.parametrize("model", ["plp", "multipeak"])
def test_linear_los_kde_equals_monte_carlo(orc, synth, rule, model):
    cat = _linear_los_catalogue(synth)
    fid = synth.FIDUCIAL if model == "plp" else synth.FIDUCIAL_MP
    shift = np.ones(len(fid))
    shift[:2] = [1.1, 0.9]
    lam = np.vstack([fid, fid * shift])
    kde = orc.loglik_kde(cat, lam, bw=rule, n_grid=256, neff_min_pixel=0.0)
    mc = orc.loglik(cat, lam, neff_min_event=0.0)
    assert np.all(np.isfinite(kde["lnL_event"]))
    # the rows are stored in float32, linear to ~6e-8 relative at the nodes
    np.testing.assert_allclose(kde["lnL_event"], mc["lnL_event"], rtol=0, atol=1e-8)
    np.testing.assert_allclose(kde["ln_xi"], mc["ln_xi"], rtol=0, atol=0)
    np.testing.assert_allclose(kde["lnL_total"], mc["lnL_total"], rtol=0, atol=1e-7)


def test_constant_los_near_the_grid_edge_is_the_truncated_kernel_mass(orc, synth):
    # one pixel with a constant LOS prior and samples near z = 0: the KDE integral of each
    # sample is the Gaussian mass inside [0, z_max], Phi((z_max - z)/h) - Phi(-z/h), so
    # L_KDE / L_MC is the w-weighted mean of that mass.  The kernels cut at z = 0 are
    # steep there, so the trapezoid error is ~1e-3 at 256 points; at 4096 it is ~5e-6,
    # while a wrong end weight would still move the result by ~2e-3
    from math import erf, sqrt
    r = np.random.default_rng(12)
    z_max = 2.0
    row = np.full(300, 1.0 / z_max, np.float32)
    ev = []
    for _ in range(80):
        dl = r.uniform(150.0, 1400.0)
        m1 = r.uniform(25.0, 60.0)
        ev.append((m1, 0.7 * m1, dl, 2.0 * np.log(dl), 0))
    inj = [(30.0, 20.0, 1000.0, -18.0), (40.0, 20.0, 2000.0, -18.0)]
    cat = tiny_catalogue(row[None, :], [ev], inj, 10.0, z_max)
    lam = synth.FIDUCIAL
    kde = orc.loglik_kde(cat, lam[None, :], n_grid=4096, neff_min_pixel=0.0)["lnL_event"][0, 0]
    mc = orc.loglik(cat, lam[None, :], neff_min_event=0.0)["lnL_event"][0, 0]
    lw = orc.ln_w_samples(lam, cat, "events")
    z = np.array([orc.z_of_x(d * lam[0] / synth.C_KMS, lam[1], z_max) for d in cat["dl"]])
    h = orc.bandwidth(z, "scott")
    Phi = lambda x: 0.5 * (1.0 + erf(x / sqrt(2.0)))
    mass = np.array([Phi((z_max - zk) / h) - Phi(-zk / h) for zk in z])
    w = np.exp(lw - lw.max())
    assert mass.min() < 0.9                       # some kernels do reach past z = 0
    assert kde - mc == pytest.approx(np.log(np.sum(w * mass) / np.sum(w)), abs=2e-5)


def test_kde_differs_from_monte_carlo_for_curved_los(orc, synth, cat_c1):
    # the smoothing is real where the LOS prior has structure (galaxy peaks)
    kde = orc.loglik_kde(cat_c1, synth.FIDUCIAL[None, :], neff_min_pixel=0.0)
    mc = orc.loglik(cat_c1, synth.FIDUCIAL[None, :], neff_min_event=0.0)
    d = np.abs(kde["lnL_event"] - mc["lnL_event"])
    assert d.max() > 1e-3 and d.max() < 1.0


def test_pixel_below_neff_threshold_is_dropped(orc, synth):
    cat = _linear_los_catalogue(synth, per_pix=(40, 60, 3))
    # pixel 2 of every event: three samples whose weights differ by e^30 (N_eff ~ 1)
    off = cat["offsets"]
    lnpe = cat["lnpe"].copy()
    for e in range(len(off) - 1):
        idx = np.arange(off[e], off[e + 1])
        p2 = idx[cat["pix"][idx] == 2]
        lnpe[p2] = cat["lnpe"][p2] + np.array([0.0, 30.0, 60.0])
    cat["lnpe"] = lnpe.astype(np.float32)
    lam = synth.FIDUCIAL[None, :]
    full = orc.loglik_kde(cat, lam, neff_min_pixel=2.0)
    kept = orc.loglik_kde(cat, lam, neff_min_pixel=0.0)
    # the same events without pixel 2, scaled back to the full sample count N_i
    keep = cat["pix"] != 2
    sub = dict(cat)
    for k in ("m1", "m2", "dl", "lnpe", "pix"):
        sub[k] = cat[k][keep]
    counts = [int(np.sum(keep[off[e]:off[e + 1]])) for e in range(len(off) - 1)]
    sub["offsets"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    ref = orc.loglik_kde(sub, lam, neff_min_pixel=0.0)
    n_full = np.diff(off)
    want = ref["lnL_event"][0] + np.log(np.array(counts) / n_full)
    np.testing.assert_allclose(full["lnL_event"][0], want, rtol=0, atol=1e-12)
    assert np.all(kept["lnL_event"][0] > full["lnL_event"][0])


def test_kde_is_permutation_invariant_and_converges_in_the_grid(orc, synth, cat_c1):
    lam = synth.FIDUCIAL[None, :]
    base = orc.loglik_kde(cat_c1, lam)
    r = np.random.default_rng(4)
    perm = dict(cat_c1)
    off = cat_c1["offsets"]
    order = np.concatenate([off[e] + r.permutation(off[e + 1] - off[e]) for e in range(len(off) - 1)])
    for k in ("m1", "m2", "dl", "lnpe", "pix"):
        perm[k] = cat_c1[k][order]
    shuffled = orc.loglik_kde(perm, lam)
    np.testing.assert_allclose(shuffled["lnL_event"], base["lnL_event"], rtol=0, atol=1e-12)
    g512 = orc.loglik_kde(cat_c1, lam, n_grid=512)["lnL_event"]
    g1024 = orc.loglik_kde(cat_c1, lam, n_grid=1024)["lnL_event"]
    fin = np.isfinite(g1024)
    assert np.abs(g512 - g1024)[fin].max() < np.abs(base["lnL_event"] - g1024)[fin].max()
