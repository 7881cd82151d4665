"""The No-U-Turn sampler driving the library: four walkers on the 10-event workload, each
transition's evaluations batched into one gwc_loglik_grad call per tree level.  Every
recorded point's log-likelihood is the FP64 oracle's there, and the walkers move."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def g(torch):
    from paper_2605_23538_gb300 import build
    build.build()
    import paper_2605_23538_gb300 as g
    return g


@pytest.mark.parametrize("model", ["plp", "multipeak"])
def test_nuts_walkers_on_the_library(torch, g, orc, synth, cat_c1, model):
    from paper_2605_23538_gb300 import nuts
    K = 4
    fid = synth.FIDUCIAL if model == "plp" else synth.FIDUCIAL_MP
    rng = np.random.default_rng(21)
    q0 = fid[None, :] * (1.0 + 0.002 * rng.standard_normal((K, len(fid))))
    inv_mass = (0.02 * np.maximum(np.abs(fid), 0.1)) ** 2
    with g.Context(cat_c1, max_K=K, mass_model=model) as ctx:
        r = nuts.sample(nuts.context_target(ctx), q0, 6, 0.05, inv_mass=inv_mass, seed=2, n_adapt=8,
                        max_depth=6)
    assert np.all(np.isfinite(r["lnL"]))
    assert np.all((r["accept_stat"] >= 0.0) & (r["accept_stat"] <= 1.0))
    assert not np.allclose(r["samples"][-1], q0)
    # the walkers shared their batches: each recorded transition took as many calls as its
    # longest walker took leapfrog steps
    np.testing.assert_array_equal(r["calls"], r["n_leapfrog"].max(axis=1))
    assert r["calls"].sum() < r["n_leapfrog"].sum()
    pts = np.stack([r["samples"][-1, 0], r["samples"][2, 3]])
    ref = orc.loglik(cat_c1, pts)["lnL_total"]
    np.testing.assert_allclose([r["lnL"][-1, 0], r["lnL"][2, 3]], ref, rtol=0, atol=1e-3)
