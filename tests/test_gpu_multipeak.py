"""GPU parity of the multi-peak mass model (App. A, Table 2) against the FP64 oracle.

The same tolerances as the power law + peak path (see test_gpu_parity.py): per-event
ln L within 1e-5, ln xi within 1e-5, total within 1e-3, the 16-component gradient within
1e-4 of its scale, flags exact; plus per-sample ln w and derivatives element by element,
the KDE form, the reduction to the single-peak context at lambda_low = 1, the one-sided
derivatives at the mixture-weight bounds, and the width and option checks.
"""
import numpy as np
import pytest

from test_gpu_parity import compare, dev

pytestmark = pytest.mark.gpu

P_LAM, P_LAM1 = 9, 15


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


@pytest.fixture(scope="module")
def lam_mp(synth):
    return np.vstack([synth.FIDUCIAL_MP, synth.lambda_batch(7, purpose=81, model="multipeak")])


@pytest.fixture(scope="module")
def cat_ragged(synth):
    # several chunks per event and ragged tails: 24 events of 300..5000 samples
    return synth.catalogue(synth.scaled("ragged", 24, ("uniform", 300, 5000), 8, 512, 30_000, "found"))


def test_c1_value_and_gradient(torch, g, orc, cat_c1, lam_mp):
    ref = orc.loglik(cat_c1, lam_mp, grad=True)
    assert ref["grad_total"].shape == (8, 16)
    with g.Context(cat_c1, max_K=8, mass_model="multipeak") as ctx:
        assert ctx.info()["n_params"] == 16
        got = ctx.loglik_grad(dev(torch, lam_mp))
        torch.cuda.synchronize()
        compare(got, ref, grad=True, label="multipeak c1 grad")
        compare(ctx.loglik(dev(torch, lam_mp)), ref, label="multipeak c1 value")


def test_ragged_catalogue_and_single_points(torch, g, orc, synth, cat_ragged):
    lam = np.vstack([synth.FIDUCIAL_MP, synth.lambda_batch(4, purpose=82, model="multipeak")])
    ref = orc.loglik(cat_ragged, lam, grad=True)
    with g.Context(cat_ragged, max_K=5, mass_model="multipeak") as ctx:
        compare(ctx.loglik_grad(dev(torch, lam)), ref, grad=True, label="multipeak ragged K=5")
        # K = 1 takes the sample-split geometry
        got = ctx.loglik_grad(dev(torch, lam[1:2]))
        compare(got, {k: v[1:2] for k, v in ref.items()}, grad=True, label="multipeak ragged K=1")


def test_lambda_low_one_is_the_single_peak_context(torch, g, synth, cat_c1):
    # lambda_low = 1 leaves the low Gaussian only: the power law + peak model at Lambda[:13]
    lam = synth.lambda_batch(4, purpose=83, model="multipeak")
    lam[:, P_LAM1] = 1.0
    with g.Context(cat_c1, max_K=4, mass_model="multipeak") as mp, g.Context(cat_c1, max_K=4) as pl:
        a = mp.loglik_grad(dev(torch, lam))
        b = pl.loglik_grad(dev(torch, lam[:, :13]))
        torch.cuda.synchronize()
    for key in ("lnL_event", "ln_xi"):
        np.testing.assert_allclose(a[key].cpu().numpy(), b[key].cpu().numpy(), rtol=0, atol=1e-5)
    ga, gb = a["grad_total"].cpu().numpy(), b["grad_total"].cpu().numpy()
    # every component of the single-peak model, lambda_g (= lambda_peak there) included;
    # d/d lambda_low at the bound is one-sided (checked against the oracle below)
    assert np.all(np.isfinite(ga))
    keep = list(range(13))
    scale = np.abs(gb[:, keep]).max(axis=0)
    np.testing.assert_allclose(ga[:, keep], gb[:, keep], rtol=1e-3, atol=1e-4 * scale.max())
    np.testing.assert_array_equal(ga[:, 13:15], 0.0)   # the absent peak's parameters


# the lambda_g and lambda_low derivatives at the mixture's bounds are one-sided: the
# oracle's forward-mode derivative of the mixture polynomial, which its tests pin
# against one-sided differences
BOUNDS = [(1.0, None), (0.0, None), (None, 1.0), (None, 0.0), (1.0, 0.0), (0.0, 1.0)]


def test_mixture_bounds_one_sided_gradient(torch, g, orc, synth, cat_c1):
    lam = np.repeat(synth.FIDUCIAL_MP[None, :], len(BOUNDS), axis=0)
    for k, (lg, ll) in enumerate(BOUNDS):
        if lg is not None:
            lam[k, P_LAM] = lg
        if ll is not None:
            lam[k, P_LAM1] = ll
    with g.Context(cat_c1, max_K=len(BOUNDS), mass_model="multipeak", neff_min_event=0.0) as ctx:
        got = ctx.loglik_grad(dev(torch, lam))
        torch.cuda.synchronize()
    ref = orc.loglik(cat_c1, lam, grad=True, neff_min_event=0.0)
    assert np.all(np.isfinite(ref["lnL_total"])) and np.all(np.isfinite(got["grad_total"].cpu().numpy()))
    out = compare(got, ref, grad=True, label="multipeak bounds")
    gg, gr = got["grad_total"].cpu().numpy(), ref["grad_total"]
    for k, b in enumerate(BOUNDS):
        print(f"bounds {b}: d/d lambda_g {gg[k, P_LAM]:.6e} (oracle {gr[k, P_LAM]:.6e}), "
              f"d/d lambda_low {gg[k, P_LAM1]:.6e} (oracle {gr[k, P_LAM1]:.6e})")
    # at lambda_g = 0 the mixture does not depend on lambda_low
    assert gg[1, P_LAM1] == 0.0 and gg[5, P_LAM1] == 0.0
    assert out["d_total"] <= 1e-3


@pytest.mark.parametrize("bound", [None, (1.0, 0.0), (0.0, 1.0)])
def test_sample_terms_elementwise(torch, g, orc, synth, cat_ragged, bound):
    # every sample's ln w and its 16 derivatives against the oracle, element by element
    # (inside the domain, and at two corners of the mixture weights)
    lam = synth.lambda_batch(1, purpose=84, model="multipeak")[0]
    if bound is not None:
        lam[P_LAM], lam[P_LAM1] = bound
    order = g.sample_order(cat_ragged)
    with g.Context(cat_ragged, max_K=1, mass_model="multipeak") as ctx:
        lnw, d, c = ctx.sample_terms(torch.tensor(lam, device="cuda"))
        c = c.cpu().numpy()
        got = lnw.cpu().numpy().astype(np.float64) + c[0]
        gd = d.cpu().numpy().T.astype(np.float64) + c[None, 1:]
    assert gd.shape[1] == 16
    ro, rg, rk = orc.ln_w_samples(lam, cat_ragged, "events", idx=order, grad=True)
    io, ig, ik = orc.ln_w_samples(lam, cat_ragged, "inj", idx=g.injection_order(cat_ragged), grad=True)
    ref, rgrad, rkink = np.concatenate([ro, io]), np.vstack([rg, ig]), np.vstack([rk, ik])
    # the samples that can move an output: within e^-30 of the largest weight of their set
    ns, off = len(order), cat_ragged["offsets"]
    rel = np.full(len(ref), -np.inf)
    for a, b in [(off[e], off[e + 1]) for e in range(len(off) - 1)] + [(ns, len(ref))]:
        r = ref[a:b]
        if np.isfinite(r).any():
            rel[a:b] = r - r[np.isfinite(r)].max()
    keep = rel > -30.0
    assert np.all(np.isfinite(got[keep])), "GPU drops a sample with non-negligible weight"
    dv = np.abs(got[keep] - ref[keep])
    assert (dv * np.exp(rel[keep])).max() <= 2e-5 and dv.max() <= 1e-3
    dg = np.abs(gd[keep] - rgrad[keep])
    tol = 2e-4 * (np.abs(rgrad[keep]) + np.abs(rgrad[keep]).mean(axis=0)[None, :]) + rkink[keep]
    bad = dg > tol
    assert bad.mean() <= 1e-3, f"{bad.sum()} derivative entries off, worst column {bad.sum(axis=0).argmax()}"


def test_kde_form(torch, g, orc, synth, cat_c1):
    lam = np.vstack([synth.FIDUCIAL_MP, synth.lambda_batch(3, purpose=85, model="multipeak")])
    ref = orc.loglik_kde(cat_c1, lam)
    with g.Context(cat_c1, max_K=4, mass_model="multipeak") as ctx:
        got = ctx.loglik_kde(dev(torch, lam))
        torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in got.items()}
    np.testing.assert_array_equal(o["flags"], ref["flags"])
    for key, tol in (("lnL_event", 1e-5), ("ln_xi", 1e-5), ("lnL_total", 1e-3)):
        fin = np.isfinite(ref[key])
        assert np.array_equal(np.isfinite(o[key]), fin)
        assert np.abs(o[key][fin] - ref[key][fin]).max(initial=0.0) <= tol, key


def test_widths_options_and_unsupported_paths(torch, g, synth, cat_c1):
    with pytest.raises(g.GwcError) as e:
        g.Context(cat_c1, max_K=1, mass_model=7)
    assert e.value.status == -1
    with g.Context(cat_c1, max_K=2, mass_model="multipeak") as ctx:
        with pytest.raises(TypeError):
            ctx.loglik(dev(torch, synth.FIDUCIAL[None, :]))       # 13 entries for a 16-entry model
        with pytest.raises(g.GwcError) as e:
            ctx.loglik_plain(dev(torch, synth.FIDUCIAL_MP[None, :]))
        assert e.value.status == -5
        # outside the domain: flag bit 0 and -inf, as for the single-peak model
        bad = synth.FIDUCIAL_MP.copy()
        bad[14] = -1.0                                           # sigma_high <= 0
        out = ctx.loglik_grad(dev(torch, np.vstack([synth.FIDUCIAL_MP, bad])))
        assert out["flags"].cpu().tolist()[1] == 1 and out["lnL_total"][1].item() == -np.inf
    with g.Context(cat_c1, max_K=1) as ctx:
        with pytest.raises(TypeError):
            ctx.loglik(dev(torch, synth.FIDUCIAL_MP[None, :]))


def test_hmc_trajectory(torch, g, orc, synth, cat_c1):
    # one recorded trajectory in the 16-dimensional space: the returned point's lnL is the
    # oracle's there
    K = 2
    with g.Context(cat_c1, max_K=K, mass_model="multipeak") as ctx:
        h = ctx.hmc(K, 4, 1e-4, np.full(16, 1e-2))
        q0 = np.vstack([synth.FIDUCIAL_MP, synth.FIDUCIAL_MP * 1.01])
        r = np.random.default_rng(7)
        h.run(q=dev(torch, q0), p=dev(torch, r.normal(size=(K, 16)) * 10.0),
              log_u=dev(torch, np.log(r.uniform(size=K))))
        torch.cuda.synchronize()
        q, lnL, acc = h.q.cpu().numpy(), h.lnL.cpu().numpy(), h.accept.cpu().tolist()
        h.close()
    assert set(acc) <= {0, 1}
    ref = orc.loglik(cat_c1, q)["lnL_total"]
    np.testing.assert_allclose(lnL, ref, rtol=0, atol=1e-3)
