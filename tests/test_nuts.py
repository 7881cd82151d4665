"""The multi-walker No-U-Turn sampler (paper_2605_23538_gb300.nuts) on targets whose
answers are known: an independent Gaussian (means, variances, a quantile, and the
adapted step size reaching the target acceptance), a strongly correlated Gaussian (the
U-turn criterion along a narrow ridge), a half-normal behind a -inf wall (points
outside the domain end their subtrees), the independence of a walker's chain from the
walkers that share its batched evaluations, and the rejection of an invalid start."""
import numpy as np
import pytest

from paper_2605_23538_gb300 import nuts


def gaussian(mean, cov):
    prec = np.linalg.inv(cov)

    def logp_grad(q):
        d = np.atleast_2d(q) - mean
        return -0.5 * np.einsum("ki,ij,kj->k", d, prec, d), -d @ prec

    return logp_grad


def test_independent_gaussian_moments_and_adaptation():
    mean, sd = np.array([1.0, -2.0, 0.5]), np.array([1.0, 0.3, 2.0])
    r = nuts.sample(gaussian(mean, np.diag(sd ** 2)), np.tile(mean, (4, 1)) + 0.1, 1000, 0.5,
                    inv_mass=sd ** 2, seed=3, n_adapt=200)
    x = r["samples"].reshape(-1, 3)
    assert np.all(np.abs(x.mean(axis=0) - mean) < 0.08 * sd)
    assert np.all(np.abs(x.std(axis=0) / sd - 1.0) < 0.08)
    z = (x[:, 0] - mean[0]) / sd[0]
    assert np.mean(z < 1.0) == pytest.approx(0.8413, abs=0.03)
    assert 0.65 < r["accept_stat"].mean() < 0.95
    # the walkers shared their batches: each recorded transition took as many calls as its
    # longest walker took leapfrog steps
    np.testing.assert_array_equal(r["calls"], r["n_leapfrog"].max(axis=1))
    assert r["calls"].sum() < r["n_leapfrog"].sum()
    assert np.all(np.isfinite(r["lnL"]))


def test_correlated_gaussian_covariance():
    cov = np.array([[1.0, 0.95], [0.95, 1.0]])
    r = nuts.sample(gaussian(np.zeros(2), cov), np.zeros((4, 2)), 1500, 0.2, seed=4, n_adapt=300)
    x = r["samples"].reshape(-1, 2)
    np.testing.assert_allclose(np.cov(x.T), cov, atol=0.12)
    assert r["depth"].mean() > 2.0                        # long trajectories along the ridge


def test_points_outside_the_domain_end_the_subtree():
    def half_normal(q):
        q = np.atleast_2d(q)
        lnL = np.where(q[:, 0] > 0.0, -0.5 * q[:, 0] ** 2, -np.inf)
        return lnL, np.where(q[:, :1] > 0.0, -q[:, :1], 0.0)
    r = nuts.sample(half_normal, np.full((4, 1), 0.5), 1500, 0.3, seed=5, n_adapt=200)
    x = r["samples"][..., 0].ravel()
    assert np.all(x > 0.0)
    assert x.mean() == pytest.approx(np.sqrt(2.0 / np.pi), abs=0.06)


def test_a_chain_does_not_depend_on_its_batch_mates():
    target = gaussian(np.zeros(3), np.diag([1.0, 4.0, 0.25]))
    q0 = np.array([[0.1, 0.2, -0.1], [1.0, -1.0, 0.3], [-0.5, 0.0, 0.2]])
    together = nuts.sample(target, q0, 30, 0.4, seed=9)
    for k in range(3):
        # walker k's stream is SeedSequence([seed, k]); run alone, give it the same one
        alone = nuts._Walker(q0[k].copy(), *[np.asarray(v)[0] for v in target(q0[k:k + 1])], 0.4,
                             np.ones(3), np.random.SeedSequence([9, k]), 10)
        for it in range(30):
            g = alone.iterate()
            req = next(g)
            while True:
                L, G = target(req[None, :])
                try:
                    req = g.send((L[0], G[0]))
                except StopIteration:
                    break
            np.testing.assert_array_equal(alone.q, together["samples"][it, k])


def test_invalid_start_is_rejected():
    def wall(q):
        q = np.atleast_2d(q)
        return np.full(len(q), -np.inf), np.zeros_like(q)
    with pytest.raises(ValueError):
        nuts.sample(wall, np.zeros((2, 2)), 5, 0.1)


def test_walkers_on_the_oracle_likelihood(orc, synth):
    # the sampler over a real 16-entry target: the FP64 oracle on a tiny catalogue, with a
    # point outside the Lambda domain (-inf) possible along the way; every recorded point
    # is in the domain and its recorded log-likelihood is the oracle's there
    from conftest import smooth_row, tiny_catalogue
    r = np.random.default_rng(6)
    ev = [[(m1, m1 * 0.7, dl, 2.0 * np.log(dl), 0) for m1, dl in zip(r.uniform(20, 40, 30), r.uniform(800, 3000, 30))]
          for _ in range(2)]
    inj = [(m1, m1 * r.uniform(0.3, 1.0), r.uniform(200, 6000), -16.0) for m1 in np.exp(r.uniform(np.log(6), np.log(120), 200))]
    cat = tiny_catalogue(smooth_row(257)[None, :], ev, inj, 800.0)

    def logp_grad(q):
        out = orc.loglik(cat, q, grad=True, neff_min_event=0.0)
        return out["lnL_total"], out["grad_total"]

    fid = synth.FIDUCIAL_MP
    res = nuts.sample(logp_grad, np.vstack([fid, fid * 1.001]), 4, 0.02,
                      inv_mass=(0.05 * np.maximum(np.abs(fid), 0.1)) ** 2, seed=1, max_depth=4)
    last = res["samples"][-1]
    assert last.shape == (2, 16) and np.all(np.isfinite(res["lnL"]))
    np.testing.assert_allclose(res["lnL"][-1], logp_grad(last)[0], rtol=0, atol=1e-12)
