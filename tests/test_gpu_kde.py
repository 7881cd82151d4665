"""GPU parity of the KDE form of the event term (gwc_loglik_kde) against the FP64 oracle.

Per-event ln L within 1e-5, ln xi within 1e-5 and the total within 1e-3 (the tolerances
of the Monte-Carlo path), the effective number of kept pixels within 1e-4 relative, flag
and finite patterns exact, for each bandwidth rule, on workloads whose (event, pixel)
groups range from one sample (dropped) to hundreds.  With LOS rows linear in z the KDE
form must also agree with the library's own Monte-Carlo path.
"""
import numpy as np
import pytest

from conftest import tiny_catalogue

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def g():
    from paper_2605_23538_gb300 import build
    build.build()
    import paper_2605_23538_gb300 as g
    return g


@pytest.fixture(scope="module")
def cat_groups(synth):
    # 24 events of 300..5000 samples over 20-pixel blocks: pixel groups of 1 to ~400
    w = synth.scaled("kde_ragged", 24, ("uniform", 300, 5000), 8, 512, 20_000, "found")
    return synth.catalogue(w)


def compare(got, ref, label):
    o = {k: v.cpu().numpy() for k, v in got.items()}
    for key in ("lnL_event", "ln_xi", "lnL_total"):
        a, b = o[key], ref[key]
        assert np.array_equal(np.isfinite(a), np.isfinite(b)), f"{label} {key} finite pattern"
    assert np.array_equal(o["flags"], ref["flags"]), f"{label} flags {o['flags']} vs {ref['flags']}"
    fin = np.isfinite(ref["lnL_event"])
    d_ev = np.abs(o["lnL_event"][fin] - ref["lnL_event"][fin]).max() if fin.any() else 0.0
    fx = np.isfinite(ref["ln_xi"])
    d_xi = np.abs(o["ln_xi"][fx] - ref["ln_xi"][fx]).max() if fx.any() else 0.0
    ft = np.isfinite(ref["lnL_total"])
    d_tot = np.abs(o["lnL_total"][ft] - ref["lnL_total"][ft]).max() if ft.any() else 0.0
    pos = ref["neff_event"] > 0
    d_nf = (np.abs(o["neff_event"][pos] - ref["neff_event"][pos]) / ref["neff_event"][pos]).max() if pos.any() else 0.0
    print(f"{label}: per-event {d_ev:.2e}, ln xi {d_xi:.2e}, total {d_tot:.2e}, kept-pixel N_eff {d_nf:.2e}")
    assert d_ev <= 1e-5 and d_xi <= 1e-5 and d_tot <= 1e-3 and d_nf <= 1e-4


@pytest.mark.parametrize("rule", ["scott", "silverman", "biweight"])
def test_kde_c1(torch, g, orc, synth, cat_c1, rule):
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(3, purpose=71)])
    ref = orc.loglik_kde(cat_c1, lam, bw=rule)
    with g.Context(cat_c1, max_K=4) as ctx:
        got = ctx.loglik_kde(torch.tensor(lam, device="cuda"), bw=rule)
        torch.cuda.synchronize()
    compare(got, ref, f"c1 {rule}")


@pytest.mark.parametrize("rule,n_grid,neff", [("scott", 256, 2.0), ("silverman", 128, 2.0),
                                              ("biweight", 256, 5.0), ("scott", 512, 0.0)])
def test_kde_ragged_groups(torch, g, orc, synth, cat_groups, rule, n_grid, neff):
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(7, purpose=72)])
    ref = orc.loglik_kde(cat_groups, lam, bw=rule, n_grid=n_grid, neff_min_pixel=neff)
    with g.Context(cat_groups, max_K=8) as ctx:
        got = ctx.loglik_kde(torch.tensor(lam, device="cuda"), bw=rule, n_grid=n_grid, neff_min_pixel=neff)
        torch.cuda.synchronize()
    compare(got, ref, f"ragged {rule} G={n_grid} neff>={neff}")


def test_kde_with_linear_los_matches_the_monte_carlo_path(torch, g, synth):
    r = np.random.default_rng(3)
    z_max, n_z = 2.0, 400
    zg = np.linspace(0.0, z_max, n_z)
    rows = []
    for j in range(3):
        a, b = 0.2 + 0.1 * j, 0.4 - 0.15 * j
        rows.append((a + b * zg) / (z_max * (a + 0.5 * b * z_max)))
    events = [[(m1, m1 * r.uniform(0.4, 0.95), dl, 2.0 * np.log(dl), j)
               for j in range(3) for m1, dl in zip(r.uniform(25, 60, 50), r.uniform(3000, 6000, 50))]
              for _ in range(3)]
    inj = [(m1, m1 * r.uniform(0.2, 1.0), r.uniform(500, 9000), -18.0)
           for m1 in np.exp(r.uniform(np.log(8.0), np.log(150.0), 400))]
    cat = tiny_catalogue(np.array(rows, np.float32), events, inj, 4000.0, z_max)
    lam = torch.tensor(np.vstack([synth.FIDUCIAL, synth.FIDUCIAL * 1.02]), device="cuda")
    with g.Context(cat, max_K=2, neff_min_event=0.0) as ctx:
        kde = ctx.loglik_kde(lam, neff_min_pixel=0.0)
        mc = ctx.loglik(lam)
        torch.cuda.synchronize()
    np.testing.assert_allclose(kde["lnL_event"].cpu().numpy(), mc["lnL_event"].cpu().numpy(), rtol=0, atol=1e-5)


def test_kde_rejects_bad_options_and_bf16_tables(torch, g, synth, cat_c1):
    lam = torch.tensor(synth.FIDUCIAL[None, :], device="cuda")
    with g.Context(cat_c1, max_K=1) as ctx:
        with pytest.raises(g.GwcError) as e:
            ctx.loglik_kde(lam, n_grid=1)
        assert e.value.status == -1
        out = g._outputs(1, ctx.n_events, lam.device, False)
        o = g.default_kde_options()
        o.bw_rule = 7
        import ctypes
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        st = g.lib().gwc_loglik_kde(ctx._ctx, 1, p(lam), ctypes.byref(o), p(out["lnL_event"]), p(out["neff_event"]),
                                    p(out["ln_xi"]), p(out["neff_sel"]), p(out["lnL_total"]), p(out["flags"]), None)
        assert st == -1
    with g.Context(cat_c1, max_K=1, los_dtype=g.LOS_BF16) as ctx:
        with pytest.raises(g.GwcError) as e:
            ctx.loglik_kde(lam)
        assert e.value.status == -5
