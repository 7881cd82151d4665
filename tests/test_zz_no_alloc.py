"""The allocation-free entry point against the context-based one.

gwc_sample_terms_noalloc serves callers that cannot allocate device memory when they
need an evaluation (inside a CUDA graph capture, or under a framework's caching
allocator): it reads caller-owned device arrays and keeps its scratch in a fixed
device array inside the library.  Here it is called twice in a row, at two different
Lambda points, and each result must match gwc_sample_terms on a context built from the
same catalogue, within the per-sample tolerance the parity tests use.  Collected last
(file name) so a failure here cannot hide the others; it also runs alone.
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


def test_noalloc_matches_context_twice(torch, synth):
    from paper_2605_23538_gb300 import build
    build.build()
    import paper_2605_23538_gb300 as g

    w = synth.scaled("noalloc", 6, ("uniform", 200, 1500), 4, 256, 4000, "found")
    cat = synth.catalogue(w)
    dev = "cuda"
    samples = torch.tensor(np.stack([cat["m1"], cat["m2"], cat["dl"], cat["lnpe"]], axis=1), device=dev)
    inj = torch.tensor(np.stack([cat["inj_m1"], cat["inj_m2"], cat["inj_dl"], cat["inj_lnpd"]], axis=1),
                       device=dev)
    pix = torch.tensor(cat["pix"], dtype=torch.int32, device=dev)
    los = torch.tensor(cat["los"], device=dev)
    order = g.sample_order(cat)
    ns = len(order)
    lams = np.vstack([synth.FIDUCIAL, synth.lambda_batch(1, purpose=21)])
    with g.Context(cat, max_K=1) as ctx:
        for lam in lams:                      # two calls in a row
            lt = torch.tensor(lam, dtype=torch.float64, device=dev)
            r_lnw, r_d, r_c = ctx.sample_terms(lt)
            n_lnw, n_d, n_c = g.sample_terms_noalloc(lt, samples, pix, inj, los, cat["z_max"])
            torch.cuda.synchronize()
            r_lnw, r_d, r_c = r_lnw.cpu().numpy(), r_d.cpu().numpy(), r_c.cpu().numpy()
            n_lnw, n_d, n_c = n_lnw.cpu().numpy(), n_d.cpu().numpy(), n_c.cpu().numpy()
            # the context orders each event's samples by (pixel, d_L) and the injections by
            # d_L; the caller's order is kept here
            perm = np.concatenate([order, ns + g.injection_order(cat)])
            n_lnw, n_d = n_lnw[perm], n_d[:, perm]
            np.testing.assert_allclose(n_c, r_c, rtol=1e-12, atol=1e-12)
            fin = np.isfinite(r_lnw)
            assert np.array_equal(fin, np.isfinite(n_lnw))
            assert fin.sum() > 1000
            assert np.max(np.abs(n_lnw[fin] - r_lnw[fin])) <= 2e-5
            scale = np.abs(r_d[:, fin]) + np.abs(r_d[:, fin]).mean(axis=1, keepdims=True)
            assert np.all(np.abs(n_d[:, fin] - r_d[:, fin]) <= 2e-4 * scale)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    import paper_2605_23538_gb300 as g
    z = torch.zeros((1, 4), dtype=torch.float32, device="cuda")
    lam = torch.zeros(13, dtype=torch.float64, device="cuda")
    los = torch.ones((1, 8), dtype=torch.float32, device="cuda")
    p = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(g.GwcError) as e:
        g.sample_terms_noalloc(lam, z, p, z, los, 2.0, n_x_table=2048)
    assert e.value.status == -1 and "scratch limit" in str(e.value)
    big = torch.ones((1, 8192), dtype=torch.float32, device="cuda")
    with pytest.raises(g.GwcError) as e:
        g.sample_terms_noalloc(lam, z, p, z, big, 2.0)
    assert e.value.status == -1 and "scratch limit" in str(e.value)


def test_noalloc_out_of_range_pixel_gets_zero_weight(torch, synth):
    # The entry point never reads the caller's pixel ids on the host, so the kernel checks
    # them: a sample whose pixel is n_pix (one past the table) or negative reads no LOS row
    # and gets w = 0, and every other sample keeps its value.
    import paper_2605_23538_gb300 as g
    w = synth.scaled("noalloc_pix", 3, ("uniform", 200, 400), 4, 256, 2000, "found")
    cat = synth.catalogue(w)
    dev = "cuda"
    samples = torch.tensor(np.stack([cat["m1"], cat["m2"], cat["dl"], cat["lnpe"]], axis=1), device=dev)
    inj = torch.tensor(np.stack([cat["inj_m1"], cat["inj_m2"], cat["inj_dl"], cat["inj_lnpd"]], axis=1),
                       device=dev)
    los = torch.tensor(cat["los"], device=dev)
    lam = torch.tensor(synth.FIDUCIAL, dtype=torch.float64, device=dev)
    pix_np = np.asarray(cat["pix"], dtype=np.int32)
    a_lnw, a_d, _ = g.sample_terms_noalloc(lam, samples, torch.tensor(pix_np, device=dev), inj, los, cat["z_max"])
    a_lnw, a_d = a_lnw.cpu().numpy(), a_d.cpu().numpy()
    fin = np.flatnonzero(np.isfinite(a_lnw[:len(pix_np)]))
    bad = fin[[0, len(fin) // 2]]
    pix_bad = pix_np.copy()
    pix_bad[bad[0]] = cat["los"].shape[0]
    pix_bad[bad[1]] = -1
    b_lnw, b_d, _ = g.sample_terms_noalloc(lam, samples, torch.tensor(pix_bad, device=dev), inj, los, cat["z_max"])
    torch.cuda.synchronize()
    b_lnw, b_d = b_lnw.cpu().numpy(), b_d.cpu().numpy()
    assert np.all(np.isneginf(b_lnw[bad])) and np.all(b_d[:, bad] == 0.0)
    rest = np.ones(len(a_lnw), bool)
    rest[bad] = False
    np.testing.assert_array_equal(b_lnw[rest], a_lnw[rest])
    np.testing.assert_array_equal(b_d[:, rest], a_d[:, rest])


def test_noalloc_replays_inside_a_cuda_graph(torch, synth):
    # The use case the entry point exists for: one warm-up call (the per-device set-up
    # runs there), then the call recorded inside the caller's own CUDA graph capture.  A
    # second Lambda copied into the captured lam tensor and a replay must give what a
    # context computes at that Lambda.
    import paper_2605_23538_gb300 as g
    w = synth.scaled("noalloc_graph", 4, ("uniform", 200, 800), 4, 256, 3000, "found")
    cat = synth.catalogue(w)
    dev = "cuda"
    samples = torch.tensor(np.stack([cat["m1"], cat["m2"], cat["dl"], cat["lnpe"]], axis=1), device=dev)
    inj = torch.tensor(np.stack([cat["inj_m1"], cat["inj_m2"], cat["inj_dl"], cat["inj_lnpd"]], axis=1),
                       device=dev)
    pix = torch.tensor(cat["pix"], dtype=torch.int32, device=dev)
    los = torch.tensor(cat["los"], device=dev)
    lam = torch.tensor(synth.FIDUCIAL, dtype=torch.float64, device=dev)
    g.sample_terms_noalloc(lam, samples, pix, inj, los, cat["z_max"])
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        n_lnw, n_d, n_c = g.sample_terms_noalloc(lam, samples, pix, inj, los, cat["z_max"])
    lam2 = synth.lambda_batch(1, purpose=22)[0]
    lam.copy_(torch.tensor(lam2, dtype=torch.float64))
    graph.replay()
    torch.cuda.synchronize()
    n_lnw, n_d, n_c = n_lnw.cpu().numpy(), n_d.cpu().numpy(), n_c.cpu().numpy()
    with g.Context(cat, max_K=1) as ctx:
        r_lnw, r_d, r_c = ctx.sample_terms(torch.tensor(lam2, dtype=torch.float64, device=dev))
        torch.cuda.synchronize()
        r_lnw, r_d, r_c = r_lnw.cpu().numpy(), r_d.cpu().numpy(), r_c.cpu().numpy()
    perm = np.concatenate([g.sample_order(cat), len(cat["pix"]) + g.injection_order(cat)])
    n_lnw, n_d = n_lnw[perm], n_d[:, perm]
    np.testing.assert_allclose(n_c, r_c, rtol=1e-12, atol=1e-12)
    fin = np.isfinite(r_lnw)
    assert np.array_equal(fin, np.isfinite(n_lnw)) and fin.sum() > 500
    assert np.max(np.abs(n_lnw[fin] - r_lnw[fin])) <= 2e-5
    scale = np.abs(r_d[:, fin]) + np.abs(r_d[:, fin]).mean(axis=1, keepdims=True)
    assert np.all(np.abs(n_d[:, fin] - r_d[:, fin]) <= 2e-4 * scale)
