"""The measurement entry points: the path census that weights the roofline's operation
counts, and the arithmetic-unit throughput probes that give its peaks.

The census runs the fused kernel's value arithmetic once per (sample, Lambda) and counts
the stages each evaluation reaches; its counts must agree exactly with what the
per-sample entry point (the same device arithmetic) reports sample by sample: the
samples whose d_L maps into [0, z_max] (a LOS cell is reported) and those with a
positive weight.
"""
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


def test_census_matches_per_sample_terms(torch, g, synth):
    w = synth.scaled("census", 12, ("uniform", 300, 3000), 8, 512, 20_000, "found")
    cat = synth.catalogue(w)
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(4, purpose=31)])
    n_total = len(cat["m1"]) + len(cat["inj_m1"])
    m1 = np.concatenate([np.asarray(cat["m1"])[g.sample_order(cat)], np.asarray(cat["inj_m1"])[g.injection_order(cat)]])
    m2 = np.concatenate([np.asarray(cat["m2"])[g.sample_order(cat)], np.asarray(cat["inj_m2"])[g.injection_order(cat)]])
    with g.Context(cat, max_K=len(lam)) as ctx:
        whole = ctx.path_census(torch.tensor(lam, device="cuda"))
        total = {k: 0 for k in whole}
        for row in lam:
            lt = torch.tensor(row, device="cuda")
            one = ctx.path_census(lt[None, :])
            lnw, _, _, cell = ctx.sample_terms(lt, grad=False, cells=True)
            lnw, cell = lnw.cpu().numpy(), cell.cpu().numpy()
            assert one["live"] == n_total
            assert one["in_range"] == int((cell >= 0).sum())
            assert one["mass_order"] == int(((cell >= 0) & (m2 <= m1)).sum())
            assert one["weight"] == int(np.isfinite(lnw).sum())
            assert (one["in_range"] >= one["mass_order"] >= one["support"] >= one["value"] >= one["weight"])
            assert one["value_win1"] <= one["value"] and one["value_win2"] <= one["value"]
            assert one["weight_win1"] <= min(one["weight"], one["value_win1"])
            assert one["weight_win2"] <= min(one["weight"], one["value_win2"])
            for k in total:
                total[k] += one[k]
        assert whole == total   # a batch counts what its points count one at a time
    print("census of the batch:", whole)


@pytest.mark.parametrize("unit", ["ffma", "ffma2", "ex2", "lg2", "rcp", "rsqrt", "dfma", "dfma_lane1"])
def test_alu_probe_runs(torch, g, unit):
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    ops = g.alu_probe(unit, 152, 200, s)
    e1.record(s)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    assert ops == 152 * 256 * 8 * 200 * {"ffma2": 2, "dfma_lane1": 1 / 32}.get(unit, 1)
    assert ms > 0.0
    print(f"{unit}: {ops / (ms / 1e3) / 1e12:.2f} Tops/s on a small launch")
    with pytest.raises(g.GwcError):
        g.alu_probe(unit, 0, 1, s)


@pytest.mark.parametrize("rule", ["scott", "biweight"])
def test_kde_census_counts(torch, g, synth, rule):
    # the KDE kernel's work counts: every event sample is evaluated once per live point in
    # the first pass; kept groups, second-pass evaluations and grid terms are bounded by
    # what they count; a batch counts what its points count one at a time
    w = synth.scaled("kde_census", 10, ("uniform", 300, 3000), 8, 512, 5_000, "found")
    cat = synth.catalogue(w)
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(3, purpose=32)])
    n_s = len(cat["m1"])
    off, pix = cat["offsets"], np.asarray(cat["pix"])
    n_groups = sum(len(np.unique(pix[off[e]:off[e + 1]])) for e in range(len(off) - 1))
    n_grid = 256
    with g.Context(cat, max_K=len(lam)) as ctx:
        whole = ctx.kde_census(torch.tensor(lam, device="cuda"), bw=rule, n_grid=n_grid)
        total = {k: 0 for k in whole}
        for row in lam:
            one = ctx.kde_census(torch.tensor(row[None, :], device="cuda"), bw=rule, n_grid=n_grid)
            assert one["pass1"] == n_s
            assert 0 < one["kept"] <= n_groups
            assert 0 < one["pass2"] <= n_s
            assert one["pass2"] <= one["terms"] <= one["pass2"] * n_grid
            for k in total:
                total[k] += one[k]
    assert whole == total
    print(f"KDE census ({rule}):", whole, f"{whole['terms'] / whole['pass2']:.1f} grid terms per sample")
