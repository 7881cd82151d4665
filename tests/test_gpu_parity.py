"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

Tolerances (from the target accuracy of the method's FP32 path):
  * per-event ln L_i: |d| <= 1e-5 absolute; total ln L: |d| <= 1e-3 absolute;
  * ln xi: |d| <= 1e-5 absolute (it is multiplied by N_det in the total);
  * N_eff (event and selection): relative 1e-4;
  * gradient: |d g| <= 1e-4 * max(|g|, 1e-2 * scale, 1e-9) + kink, where scale is the size of
    the per-sample derivatives whose weighted difference the gradient is (returned by
    the oracle): near the likelihood peak the total gradient is a small difference of
    large terms that no FP32 evaluation resolves to 1e-4 of itself; and kink (also from
    the oracle) bounds the difference between the two one-sided derivatives of the
    piecewise-linear LOS prior for samples within 2e-5 cells of a grid node, where the
    FP32 position (accurate to ~1e-6 cells) may fall on the other side of the node and
    either side is correct;
  * flags and the finite/-inf pattern: exact.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_EVENT, TOL_TOTAL, TOL_XI, TOL_NEFF, TOL_GRAD = 1e-5, 1e-3, 1e-5, 1e-4, 1e-4


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


def dev(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device="cuda")


def compare(got, ref, grad=False, label=""):
    ge = got["lnL_event"].cpu().numpy()
    re_ = ref["lnL_event"]
    assert np.array_equal(np.isfinite(ge), np.isfinite(re_)), f"{label}: finite pattern"
    fin = np.isfinite(re_)
    d_ev = np.max(np.abs(ge[fin] - re_[fin]), initial=0.0)
    assert d_ev <= TOL_EVENT, f"{label}: per-event |d| = {d_ev}"
    np.testing.assert_array_equal(got["flags"].cpu().numpy(), ref["flags"], err_msg=label)
    gx = got["ln_xi"].cpu().numpy()
    fx = np.isfinite(ref["ln_xi"])
    assert np.array_equal(np.isfinite(gx), fx)
    d_xi = np.max(np.abs(gx[fx] - ref["ln_xi"][fx]), initial=0.0)
    assert d_xi <= TOL_XI, f"{label}: ln xi |d| = {d_xi}"
    gt = got["lnL_total"].cpu().numpy()
    ft = np.isfinite(ref["lnL_total"])
    assert np.array_equal(np.isfinite(gt), ft)
    d_tot = np.max(np.abs(gt[ft] - ref["lnL_total"][ft]), initial=0.0)
    assert d_tot <= TOL_TOTAL, f"{label}: total |d| = {d_tot}"
    ne = got["neff_event"].cpu().numpy()
    ok = ref["neff_event"] > 0
    np.testing.assert_allclose(ne[ok], ref["neff_event"][ok], rtol=TOL_NEFF)
    np.testing.assert_allclose(got["neff_sel"].cpu().numpy(), ref["neff_sel"], rtol=TOL_NEFF)
    out = dict(d_event=d_ev, d_xi=d_xi, d_total=d_tot)
    if grad:
        gg = got["grad_total"].cpu().numpy()
        gr, sc, kink = ref["grad_total"], ref["grad_scale"], ref["grad_kink"]
        rel = np.maximum(np.abs(gg - gr) - kink, 0.0) / np.maximum(np.maximum(np.abs(gr), 1e-2 * sc), 1e-9)
        rel[~ft] = 0.0
        assert np.all(rel <= TOL_GRAD), f"{label}: grad rel err {rel.max()} at {np.unravel_index(rel.argmax(), rel.shape)}"
        out["grad_rel"] = float(rel.max())
        out["kink_used"] = int(np.count_nonzero((np.abs(gg - gr) > 1e-4 * np.maximum(np.abs(gr), 1e-2 * sc)) & (kink > 0)))
        # the plain relative error of each finite component, and how many components pass
        # only through the 1e-2 x scale floor (|d| > 1e-4 |g| where |g| < 1e-2 scale)
        plain = np.abs(gg - gr)[ft] / np.maximum(np.abs(gr[ft]), 1e-300)
        out["grad_plain_rel_max"] = float(plain.max()) if plain.size else 0.0
        out["floor_used"] = int(np.count_nonzero(((np.abs(gr) < 1e-2 * sc) & (np.abs(gg - gr) > TOL_GRAD * np.abs(gr)))[ft]))
    print(label, out)
    return out


@pytest.fixture(scope="module")
def cat_c1(synth):
    return synth.catalogue("c1")


@pytest.fixture(scope="module")
def lam_c1(synth):
    return np.vstack([synth.FIDUCIAL, synth.lambda_batch(7, purpose=11)])


def test_c1_value_and_gradient(torch, g, orc, cat_c1, lam_c1):
    ref = orc.loglik(cat_c1, lam_c1, grad=True)
    with g.Context(cat_c1, max_K=8) as ctx:
        got = ctx.loglik_grad(dev(torch, lam_c1))
        torch.cuda.synchronize()
        compare(got, ref, grad=True, label="c1 grad")
        val = ctx.loglik(dev(torch, lam_c1))
        compare(val, ref, label="c1 value")
        # the value and value+gradient passes agree to the last bit on the value
        assert torch.equal(val["lnL_total"], got["lnL_total"]) or \
            np.allclose(val["lnL_total"].cpu().numpy(), got["lnL_total"].cpu().numpy(), atol=1e-9)


def test_c1_each_lambda_alone(torch, g, orc, cat_c1, lam_c1):
    # K = 1 uses the sample-split geometry (8 warps on one Lambda)
    ref = orc.loglik(cat_c1, lam_c1[:3], grad=True)
    with g.Context(cat_c1, max_K=8) as ctx:
        for k in range(3):
            got = ctx.loglik_grad(dev(torch, lam_c1[k:k + 1]))
            r = {key: v[k:k + 1] for key, v in ref.items()}
            compare(got, r, grad=True, label=f"c1 K=1 #{k}")


@pytest.mark.parametrize("K", [2, 3, 5])
def test_c1_small_batches(torch, g, orc, cat_c1, lam_c1, K):
    # batches of fewer than 8 points split each point's samples over 8/K warps (the
    # largest power of two: 4 at K = 2, 2 at K = 3, 1 at K = 5); each shape against the oracle
    ref = orc.loglik(cat_c1, lam_c1[:K], grad=True)
    with g.Context(cat_c1, max_K=8) as ctx:
        got = ctx.loglik_grad(dev(torch, lam_c1[:K]))
        compare(got, ref, grad=True, label=f"c1 K={K}")


@pytest.fixture(scope="module")
def cat_ragged(synth):
    # several chunks per event and ragged tails: 24 events of 300..5000 samples
    w = synth.scaled("ragged", 24, ("uniform", 300, 5000), 8, 512, 30_000, "found")
    return synth.catalogue(w)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_sample_terms_elementwise(torch, g, orc, synth, cat_ragged, which):
    # every sample's ln w and its 13 derivatives against the oracle, element by element
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(9, purpose=13)[:1],
                     synth.lambda_batch(1, purpose=16)])[which]
    order = g.sample_order(cat_ragged)
    with g.Context(cat_ragged, max_K=1) as ctx:
        lnw, d, c = ctx.sample_terms(torch.tensor(lam, device="cuda"))
        c = c.cpu().numpy()
        got = lnw.cpu().numpy().astype(np.float64) + c[0]
        gd = d.cpu().numpy().T.astype(np.float64) + c[None, 1:]
    ro, rg, rk = orc.ln_w_samples(lam, cat_ragged, "events", idx=order, grad=True)
    io, ig, ik = orc.ln_w_samples(lam, cat_ragged, "inj", idx=g.injection_order(cat_ragged), grad=True)
    ref, rgrad, rkink = np.concatenate([ro, io]), np.vstack([rg, ig]), np.vstack([rk, ik])
    # only samples whose weight is within e^-30 of the largest in their set (their event,
    # or the injections) can move any output; below that FP32 cannot resolve terms such
    # as ln S = -delta_m/m' for m' of a few ulp, and the weight is irrelevant anyway
    ns = len(order)
    off = cat_ragged["offsets"]
    rel = np.full(len(ref), -np.inf)
    for a, b in [(off[e], off[e + 1]) for e in range(len(off) - 1)] + [(ns, len(ref))]:
        r = ref[a:b]
        if np.isfinite(r).any():
            rel[a:b] = r - r[np.isfinite(r)].max()
    keep = rel > -30.0
    gfin = np.isfinite(got)
    assert np.all(gfin[keep]), "GPU drops a sample with non-negligible weight"
    gl = np.where(gfin, got, -np.inf)
    for a, b in [(off[e], off[e + 1]) for e in range(len(off) - 1)] + [(ns, len(ref))]:
        seg = gl[a:b]
        if np.isfinite(seg).any():
            gl[a:b] = seg - seg[np.isfinite(seg)].max()
    assert np.all(gl[~keep & gfin] < -25.0), "GPU gives weight to a sample the oracle says is negligible"
    dv = np.abs(got[keep] - ref[keep])
    # each relevant weight to 2e-5 of its set's largest weight, and no gross error anywhere
    wv = dv * np.exp(rel[keep])
    assert wv.max() <= 2e-5, f"per-sample weight error max {wv.max()} (ln w |d| p99 {np.percentile(dv, 99)})"
    assert dv.max() <= 1e-3, f"per-sample ln w |d| max {dv.max()}"
    dg = np.abs(gd[keep] - rgrad[keep])
    tol = 2e-4 * (np.abs(rgrad[keep]) + np.abs(rgrad[keep]).mean(axis=0)[None, :]) + rkink[keep]
    bad = dg > tol
    print(f"terms Lambda#{which}: {keep.sum()} of {len(ref)} relevant; value max {dv.max():.2e} "
          f"weighted max {wv.max():.2e} "
          f"p99 {np.percentile(dv, 99):.2e}; grad worst ratio {(dg / tol).max():.2e}; "
          f"kink samples {int((rkink[keep] > 0).any(axis=1).sum())}")
    assert not bad.any(), f"{bad.sum()} gradient elements outside tolerance, e.g. {np.argwhere(bad)[:5]}"


def test_batch_of_64_ragged(torch, g, orc, synth, cat_ragged):
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(63, purpose=12)])
    ref = orc.loglik(cat_ragged, lam)
    with g.Context(cat_ragged, max_K=64, chunk=1024) as ctx:
        got = ctx.loglik(dev(torch, lam))
        compare(got, ref, label="ragged K=64")


def test_batch_gradient_ragged(torch, g, orc, synth, cat_ragged):
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(9, purpose=13)])
    ref = orc.loglik(cat_ragged, lam, grad=True)
    with g.Context(cat_ragged, max_K=16, chunk=512, lambda_tile=8) as ctx:
        got = ctx.loglik_grad(dev(torch, lam))
        compare(got, ref, grad=True, label="ragged grad K=10")


@pytest.mark.parametrize("chunk,tile,group", [(64, 1, 1), (256, 3, 8), (4096, 40, 4), (1024, 16, 1)])
def test_tiling_does_not_change_results(torch, g, synth, cat_ragged, chunk, tile, group):
    lam = dev(torch, np.vstack([synth.FIDUCIAL, synth.lambda_batch(11, purpose=14)]))
    with g.Context(cat_ragged, max_K=16) as a, g.Context(cat_ragged, max_K=16, chunk=chunk,
                                                         lambda_tile=tile, lambda_group=group) as b:
        ra, rb = a.loglik_grad(lam), b.loglik_grad(lam)
        ea, eb = ra["lnL_event"].cpu().numpy(), rb["lnL_event"].cpu().numpy()
        fin = np.isfinite(ea)
        assert np.array_equal(fin, np.isfinite(eb))
        assert np.max(np.abs(ea[fin] - eb[fin])) < 2e-6
        assert np.allclose(ra["grad_total"].cpu().numpy(), rb["grad_total"].cpu().numpy(), rtol=1e-4, atol=1e-3)


def test_deterministic(torch, g, synth, cat_ragged):
    lam = dev(torch, synth.lambda_batch(16, purpose=15))
    with g.Context(cat_ragged, max_K=16) as ctx:
        a = ctx.loglik_grad(lam)
        b = ctx.loglik_grad(lam)
        for k in a:
            assert torch.equal(a[k], b[k]) or torch.equal(torch.nan_to_num(a[k]), torch.nan_to_num(b[k])), k


def test_plain_path_matches(torch, g, orc, synth, cat_c1, lam_c1):
    ref = orc.loglik(cat_c1, lam_c1[:4], grad=True)
    with g.Context(cat_c1, max_K=8) as ctx:
        got = ctx.loglik_plain(dev(torch, lam_c1[:4]), grad=True)
        compare(got, ref, grad=True, label="plain")
        val = ctx.loglik_plain(dev(torch, lam_c1[:4]), grad=False)
        compare(val, ref, label="plain value")


def test_host_entry_point(torch, g, synth, cat_c1, lam_c1):
    with g.Context(cat_c1, max_K=8) as ctx:
        d = ctx.loglik_grad(dev(torch, lam_c1))
        tot, flags, grad = ctx.loglik_grad_host(lam_c1)
        np.testing.assert_array_equal(tot, d["lnL_total"].cpu().numpy())
        np.testing.assert_array_equal(flags, d["flags"].cpu().numpy())
        np.testing.assert_array_equal(grad, d["grad_total"].cpu().numpy())


def test_autograd_function(torch, g, cat_c1, lam_c1):
    with g.Context(cat_c1, max_K=8) as ctx:
        lam = dev(torch, lam_c1[:3]).requires_grad_(True)
        tot = g.GwcLogLik.apply(lam, ctx)
        w = torch.tensor([0.5, -1.0, 2.0], dtype=torch.float64, device="cuda")
        (tot * w).sum().backward()
        ref = ctx.loglik_grad(lam.detach())["grad_total"] * w[:, None]
        assert torch.allclose(lam.grad, ref)


def test_los_cell_index_bit_exact(torch, g, orc):
    rng = np.random.default_rng(3)
    for nz, zmax in ((512, 2.0), (2048, 2.0), (1000, 1.7), (2, 0.3)):
        z = rng.uniform(-0.1, zmax * 1.05, 4000).astype(np.float32)
        # values on and next to every 37th grid node, in float32
        nodes = (np.arange(0, nz, 37) * (zmax / (nz - 1))).astype(np.float32)
        z = np.concatenate([z, nodes, np.nextafter(nodes, np.float32(-1)), np.nextafter(nodes, np.float32(9)),
                            np.float32([0.0, zmax, -0.0])])
        got = g.los_cell_index(torch.tensor(z, device="cuda"), nz, zmax).cpu().numpy()
        ref = np.array([orc.los_cell(v, nz, zmax) for v in z], dtype=np.int32)
        np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_fused_kernel_cell_index_against_oracle(torch, g, orc, synth, cat_ragged, which):
    # The LOS cell each sample is interpolated in, as the likelihood kernels compute it
    # (their own position arithmetic, reported through gwc_sample_terms), against the
    # oracle's floor of the exact grid position z (n_z - 1) / z_max: equal for every sample
    # except within NODE_WINDOW cells of a node, where either neighbouring cell gives the
    # same value; those are counted.
    from conftest import cell_mismatches
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(9, purpose=13)[:1],
                     synth.lambda_batch(1, purpose=16)])[which]
    nz, zmax = cat_ragged["los"].shape[1], float(cat_ragged["z_max"])
    with g.Context(cat_ragged, max_K=1) as ctx:
        *_, cell = ctx.sample_terms(torch.tensor(lam, device="cuda"), grad=False, cells=True)
        cell = cell.cpu().numpy()
    dl = np.concatenate([np.asarray(cat_ragged["dl"])[g.sample_order(cat_ragged)],
                         np.asarray(cat_ragged["inj_dl"])[g.injection_order(cat_ragged)]])
    rc, rp = orc.sample_cells(lam, dl, nz, zmax)
    n, near, diff = cell_mismatches(cell, rc, rp)
    print(f"cells Lambda#{which}: {n} samples in range, {near} within {2e-5} cells of a node, "
          f"{diff} of those in the neighbouring cell")
    assert n > 20_000


def test_pixel_ids_used_verbatim(torch, g, orc, synth, cat_c1):
    # shifting every sample to another block of pixels changes results exactly as the
    # oracle says (a pixel mix-up would not)
    cat = dict(cat_c1)
    cat["pix"] = ((cat_c1["pix"].astype(np.int64) + 101) % cat_c1["los"].shape[0]).astype(np.int32)
    lam = np.vstack([synth.FIDUCIAL])
    ref = orc.loglik(cat, lam, neff_min_event=0.0)
    with g.Context(cat, max_K=1, neff_min_event=0.0) as ctx:
        compare(ctx.loglik(dev(torch, lam)), ref, label="shifted pixels")


def test_edge_lambdas(torch, g, orc, synth, cat_c1):
    base = synth.FIDUCIAL
    pts = []
    for idx, v in ((9, 0.0), (9, 1.0), (6, 0.0), (2, 1.0), (3, -1.0), (3, -1.0005), (1, 0.0), (1, 1.0)):
        p = base.copy()
        p[idx] = v
        pts.append(p)
    bad = base.copy()
    bad[5] = 4.0          # m_max < m_min: outside the domain
    pts.append(bad)
    nan = base.copy()
    nan[0] = np.nan
    pts.append(nan)
    lam = np.vstack(pts)
    ref = orc.loglik(cat_c1, lam, grad=True, neff_min_event=0.0)
    with g.Context(cat_c1, max_K=16, neff_min_event=0.0) as ctx:
        got = ctx.loglik_grad(dev(torch, lam))
        compare(got, ref, grad=True, label="edges")
        fl = got["flags"].cpu().numpy()
        assert fl[-1] == 1 and fl[-2] == 1
        assert got["lnL_total"][-1].item() == -math.inf


def test_event_beyond_the_grid_and_thresholds(torch, g, orc, synth, cat_c1):
    cat = dict(cat_c1)
    cat["dl"] = cat_c1["dl"].copy()
    cat["dl"][: cat_c1["offsets"][1]] = np.float32(1e6)   # event 0 entirely beyond z_max
    lam = np.vstack([synth.FIDUCIAL])
    for nmin, smin in ((2.0, 0.0), (0.0, 0.0), (0.0, 1e12)):
        ref = orc.loglik(cat, lam, neff_min_event=nmin, neff_min_sel=smin)
        with g.Context(cat, max_K=1, neff_min_event=nmin, neff_min_sel=smin) as ctx:
            got = ctx.loglik(dev(torch, lam))
            compare(got, ref, label=f"thresholds {nmin} {smin}")
            assert got["lnL_total"][0].item() == -math.inf


def test_single_event_single_sample_and_tiny_inputs(torch, g, orc, synth):
    from conftest import tiny_catalogue
    cat = tiny_catalogue([[0.5, 0.5]], [[(45.0, 30.0, 2500.0, 15.7, 0)]],
                         [(50.0, 40.0, 3000.0, -18.0)], n_draw=3.0)
    lam = np.vstack([synth.FIDUCIAL])
    ref = orc.loglik(cat, lam, neff_min_event=0.0)
    with g.Context(cat, max_K=1, neff_min_event=0.0) as ctx:
        compare(ctx.loglik(dev(torch, lam)), ref, label="tiny")


def test_no_events(torch, g, synth, cat_c1):
    cat = synth.subset_events(cat_c1, [])
    with g.Context(cat, max_K=2) as ctx:
        out = ctx.loglik(dev(torch, np.vstack([synth.FIDUCIAL] * 2)))
        assert out["lnL_total"].cpu().numpy().tolist() == [0.0, 0.0]


def test_compensated_and_bf16_variants(torch, g, orc, synth, cat_c1, lam_c1):
    ref = orc.loglik(cat_c1, lam_c1)
    with g.Context(cat_c1, max_K=8, accum=1) as ctx:
        compare(ctx.loglik(dev(torch, lam_c1)), ref, label="compensated")
    with g.Context(cat_c1, max_K=8, los_dtype=1) as ctx:
        got = ctx.loglik(dev(torch, lam_c1))
        d = np.nanmax(np.abs(got["lnL_event"].cpu().numpy() - ref["lnL_event"]))
        assert d < 1e-2   # bfloat16 rows carry 8 significand bits: an error study, not parity
        print("bf16 LOS: max per-event |d| =", d)


def test_invalid_calls(torch, g, synth, cat_c1):
    with g.Context(cat_c1, max_K=2) as ctx:
        with pytest.raises(g.GwcError):
            ctx.loglik(dev(torch, np.vstack([synth.FIDUCIAL] * 3)))   # K > max_K
        with pytest.raises(TypeError):
            ctx.loglik(torch.zeros((1, 13), dtype=torch.float32, device="cuda"))


def test_cap_per_pixel_matches_the_oracle_on_the_capped_catalogue(torch, g, orc, synth, cat_ragged):
    # the library's random per-pixel cap and the same choice made in numpy must give the
    # same catalogue: compare both paths against the oracle on the capped catalogue
    cap, seed = 40, 2024
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(5, purpose=81)])
    small = g.capped(cat_ragged, cap, seed)
    assert len(small["m1"]) < len(cat_ragged["m1"])
    ref = orc.loglik(small, lam, grad=True)
    with g.Context(cat_ragged, max_K=6, cap_per_pixel=cap, cap_seed=seed) as ctx:
        assert ctx.info()["n_samples"] == len(small["m1"])
        got = ctx.loglik_grad(dev(torch, lam))
        kde = ctx.loglik_kde(dev(torch, lam))
    compare(got, ref, grad=True, label=f"cap {cap}")
    kref = orc.loglik_kde(small, lam)
    fin = np.isfinite(kref["lnL_event"])
    d = np.abs(kde["lnL_event"].cpu().numpy()[fin] - kref["lnL_event"][fin]).max()
    assert d <= 1e-5, d


def test_spectral_siren_single_uniform_row(torch, g, orc, synth, cat_c1):
    # spectral-siren mode: one LOS row, uniform in comoving volume, for every sample
    z_max = float(cat_c1["z_max"])
    z = np.linspace(0.0, z_max, 512)
    E = np.sqrt(0.3 * (1 + z) ** 3 + 0.7)
    dc = np.concatenate([[0.0], np.cumsum(0.5 * (1 / E[1:] + 1 / E[:-1]) * np.diff(z))])
    row = dc ** 2 / E
    row /= np.sum(0.5 * (row[1:] + row[:-1]) * np.diff(z))
    cat = dict(cat_c1)
    cat["los"] = row[None, :].astype(np.float32)
    cat["pix"] = np.zeros_like(cat_c1["pix"])
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(3, purpose=82)])
    ref = orc.loglik(cat, lam, grad=True)
    with g.Context(cat, max_K=4) as ctx:
        got = ctx.loglik_grad(dev(torch, lam))
    compare(got, ref, grad=True, label="spectral siren")


def test_event_shards_merge_to_the_full_likelihood(torch, g, orc, synth, cat_ragged):
    # two contexts on one GPU, each with half of the events and half of the injections
    # (and the whole n_draw), combined by shard.merge_parts; compared with the oracle on the
    # whole catalogue exactly as a single context would be
    from paper_2605_23538_gb300 import shard
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(5, purpose=83)])
    ref = orc.loglik(cat_ragged, lam, grad=True)
    ne, ni = len(cat_ragged["offsets"]) - 1, len(cat_ragged["inj_m1"])
    halves = []
    for ev, (a, b) in (([*range(0, ne // 2)], (0, ni // 2)), ([*range(ne // 2, ne)], (ni // 2, ni))):
        part = synth.subset_events(cat_ragged, ev)
        for k in ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd"):
            part[k] = cat_ragged[k][a:b]
        halves.append(part)
    parts = []
    for part in halves:
        with g.Context(part, max_K=6, neff_min_sel=0.0) as ctx:
            parts.append(ctx.loglik_parts(dev(torch, lam)))
    merged = shard.merge_parts(parts)
    got = {"lnL_event": torch.cat([p["lnL_event"] for p in parts], dim=1),
           "neff_event": torch.cat([p["neff_event"] for p in parts], dim=1)}
    for k in ("lnL_total", "ln_xi", "neff_sel", "flags", "grad_total"):
        got[k] = torch.as_tensor(merged[k])
    compare(got, ref, grad=True, label="two event shards")
