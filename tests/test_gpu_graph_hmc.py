"""Recorded calls (gwc_graph) and the recorded HMC trajectory (gwc_hmc), through the C ABI.

A graph replay must give bit-identical outputs to a direct call on the same Lambda
batch: the same three kernels run with the same geometry, every (item, Lambda) partial
is reduced in a fixed order whichever persistent CTA takes it, and the merge is
deterministic.  The trajectory is checked against the definition of the leapfrog
integrator run on the host with the oracle's FP64 gradient, for exact time reversal
(negating the final momenta retraces the path), for a bounded energy error, and for
the Metropolis decision and the handling of chains that leave the domain.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# per-parameter scales for the trajectory tests (about the spread of the c1 likelihood
# near the fiducial point, from its curvature); M^-1 = diag(SCALE^2)
SCALE = np.array([2.0, 0.1, 0.5, 0.5, 0.5, 5.0, 0.5, 2.0, 1.0, 0.02, 0.5, 2.0, 0.5])


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
def cat_graph(synth):
    w = synth.scaled("graph", 12, ("uniform", 300, 3000), 8, 512, 20_000, "found")
    return synth.catalogue(w)


def _equal(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    same = (a == b) | (np.isnan(a) & np.isnan(b))
    return bool(same.all())


@pytest.mark.parametrize("grad", [True, False])
def test_graph_replay_is_bit_identical_to_direct_calls(torch, g, synth, cat_graph, grad):
    K = 16
    batches = [synth.lambda_batch(K, purpose=31), synth.lambda_batch(K, purpose=32)]
    batches[1][3] = synth.FIDUCIAL
    with g.Context(cat_graph, max_K=K) as ctx:
        lam = torch.empty((K, 13), dtype=torch.float64, device="cuda")
        graph = ctx.graph(lam, grad=grad)
        for b in batches:
            lt = torch.tensor(b, dtype=torch.float64, device="cuda")
            direct = ctx.loglik_grad(lt) if grad else ctx.loglik(lt)
            lam.copy_(lt)
            rep = graph.launch()
            torch.cuda.synchronize()
            for key in direct:
                assert _equal(direct[key], rep[key]), key
        graph.close()


def test_call_inside_torch_graph_capture(torch, g, synth, cat_graph):
    # the per-call path allocates nothing and never synchronises, so a caller's own
    # stream capture can record it
    K = 8
    with g.Context(cat_graph, max_K=K) as ctx:
        lam = torch.tensor(synth.lambda_batch(K, purpose=33), dtype=torch.float64, device="cuda")
        out = g._outputs(K, ctx.n_events, lam.device, True)
        ref = ctx.loglik_grad(lam.clone())
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            g.loglik_grad(ctx._ctx, lam, ctx.n_events, side, out)   # warm-up outside capture
        torch.cuda.current_stream().wait_stream(side)
        cg = torch.cuda.CUDAGraph()
        with torch.cuda.graph(cg):
            g.loglik_grad(ctx._ctx, lam, ctx.n_events, torch.cuda.current_stream(), out)
        for v in out.values():
            v.zero_()
        cg.replay()
        torch.cuda.synchronize()
        for key in ref:
            assert _equal(ref[key], out[key]), key


def test_graph_after_context_destroyed_is_rejected(torch, g, synth, cat_graph):
    ctx = g.Context(cat_graph, max_K=2)
    lam = torch.tensor(synth.lambda_batch(2, purpose=34), dtype=torch.float64, device="cuda")
    graph = ctx.graph(lam, grad=False)
    graph.launch()
    torch.cuda.synchronize()
    ctx.close()
    with pytest.raises(g.GwcError) as e:
        graph.launch()
    assert e.value.status == -1
    graph.close()


def _start(synth, K, seed):
    r = np.random.default_rng(seed)
    q = synth.FIDUCIAL[None, :] * (1.0 + 0.01 * r.standard_normal((K, 13)))
    p = r.standard_normal((K, 13)) / SCALE[None, :]        # p ~ N(0, M), M = diag(1/SCALE^2)
    return q, p


def _hmc(torch, g, ctx, K, L, eps):
    return ctx.hmc(K, L, np.full(K, eps), SCALE ** 2)


def _np(t):
    return t.detach().cpu().numpy().copy()


def test_hmc_matches_host_leapfrog_with_oracle_gradient(torch, g, orc, synth, cat_c1):
    K, L, eps = 3, 8, 0.02
    q0, p0 = _start(synth, K, 1)
    with g.Context(cat_c1, max_K=K) as ctx:
        h = _hmc(torch, g, ctx, K, L, eps)
        h.run(torch.tensor(q0, device="cuda"), torch.tensor(p0, device="cuda"),
              torch.full((K,), -np.inf, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        q_gpu, p_gpu, H_gpu, acc = _np(h.q), _np(h.p), _np(h.H), _np(h.accept)
        h.close()
    # the integrator written out on the host with the FP64 oracle's gradient
    im = SCALE ** 2
    q, p = q0.copy(), p0.copy()
    r = orc.loglik(cat_c1, q, grad=True)
    H0 = -r["lnL_total"] + 0.5 * (p * p * im).sum(1)
    for step in range(L):
        p = p + 0.5 * eps * r["grad_total"]
        q = q + eps * im * p
        r = orc.loglik(cat_c1, q, grad=True)
        p = p + 0.5 * eps * r["grad_total"]
    H1 = -r["lnL_total"] + 0.5 * (p * p * im).sum(1)
    assert np.all(acc == 1)
    dq = np.abs(q_gpu - q) / SCALE[None, :]
    dp = np.abs(p_gpu - p) * SCALE[None, :]
    print(f"hmc vs oracle leapfrog: max |dq|/scale {dq.max():.2e}, |dp| scale {dp.max():.2e}, "
          f"H0 {H_gpu[:, 0] - H0}, H1 {H_gpu[:, 1] - H1}")
    assert dq.max() <= 1e-4 and dp.max() <= 1e-3
    np.testing.assert_allclose(H_gpu[:, 0], H0, rtol=0, atol=1e-3)
    np.testing.assert_allclose(H_gpu[:, 1], H1, rtol=0, atol=1e-3)


def test_hmc_trajectory_reverses_and_bounds_energy_error(torch, g, synth, cat_c1):
    # The likelihood is only piecewise smooth: the LOS prior is linear between grid nodes,
    # so the gradient jumps where a sample's z crosses a node, and the leapfrog energy
    # error falls like eps rather than eps^2 (the host integrator with the oracle's
    # gradient gives |H1 - H0| up to 0.28 at eps = 0.02 for these chains; the GPU gives
    # up to 0.075 at 0.005).  The energy check is a bound against blow-up; the match to
    # the oracle's integrator is tested above.
    K, L, eps = 4, 32, 0.005
    q0, p0 = _start(synth, K, 2)
    with g.Context(cat_c1, max_K=K) as ctx:
        h = _hmc(torch, g, ctx, K, L, eps)
        always = torch.full((K,), -np.inf, dtype=torch.float64, device="cuda")
        h.run(torch.tensor(q0, device="cuda"), torch.tensor(p0, device="cuda"), always)
        torch.cuda.synchronize()
        q1, p1, H = _np(h.q), _np(h.p), _np(h.H)
        assert np.all(_np(h.accept) == 1)
        assert np.all(np.abs(H[:, 1] - H[:, 0]) < 0.5), H
        # a replay with the same inputs is bit-identical
        h.run(torch.tensor(q0, device="cuda"), torch.tensor(p0, device="cuda"), always)
        torch.cuda.synchronize()
        assert np.array_equal(_np(h.q), q1) and np.array_equal(_np(h.p), p1)
        # negated momenta retrace the path back to the start
        h.run(torch.tensor(q1, device="cuda"), torch.tensor(-p1, device="cuda"), always)
        torch.cuda.synchronize()
        q2, p2 = _np(h.q), _np(h.p)
        h.close()
    assert np.max(np.abs(q2 - q0) / SCALE[None, :]) <= 1e-9
    assert np.max(np.abs(p2 + p0) * SCALE[None, :]) <= 1e-9


def test_hmc_metropolis_decision_and_domain_exit(torch, g, synth, cat_c1):
    K, L, eps = 3, 32, 0.02
    q0, p0 = _start(synth, K, 3)
    # chain 2 starts next to lambda_peak = 0 with a momentum that carries it below 0
    q0[2, 9] = 0.002
    p0[2, 9] = -40.0 / SCALE[9]
    with g.Context(cat_c1, max_K=K) as ctx:
        ref = ctx.loglik_grad(torch.tensor(q0, device="cuda"))
        h = _hmc(torch, g, ctx, K, L, eps)
        never = torch.full((K,), np.inf, dtype=torch.float64, device="cuda")
        h.run(torch.tensor(q0, device="cuda"), torch.tensor(p0, device="cuda"), never)
        torch.cuda.synchronize()
        # rejected: the start comes back with its own log-likelihood and gradient
        assert np.all(_np(h.accept) == 0)
        assert np.array_equal(_np(h.q), q0)
        assert _equal(h.lnL, ref["lnL_total"]) and _equal(h.grad, ref["grad_total"])
        always = torch.full((K,), -np.inf, dtype=torch.float64, device="cuda")
        h.run(torch.tensor(q0, device="cuda"), torch.tensor(p0, device="cuda"), always)
        torch.cuda.synchronize()
        acc, H = _np(h.accept), _np(h.H)
        h.close()
    # the chain that left the domain is rejected and returned unchanged; the others accept
    assert acc.tolist() == [1, 1, 0]
    assert np.isinf(H[2, 1])


def test_autotune_picks_a_timed_shape_and_keeps_parity(torch, g, orc, synth, cat_graph):
    # tuning re-splits the work items (chunk 2048 -> 1024 -> 2048 -> the choice), and the
    # plain path's per-sample item map with them; both paths must still match the oracle
    K = 24
    lam = np.vstack([synth.FIDUCIAL, synth.lambda_batch(K - 1, purpose=35)])
    ref = orc.loglik(cat_graph, lam)
    lt = torch.tensor(lam, dtype=torch.float64, device="cuda")
    with g.Context(cat_graph, max_K=K, chunk=2048) as ctx:
        graph = ctx.graph(lt.clone(), grad=False)
        with pytest.raises(g.GwcError) as e:           # recorded launches hold the layout
            ctx.autotune(lt)
        assert e.value.status == -1
        graph.close()
        ctx.loglik_plain(lt[:2])                       # plain-path scratch exists before the re-split
        r = ctx.autotune(lt)
        # tiles 16 .. 256 clamp to 16, 24, 24, 24, 24 at K = 24: 3 chunks x 2 tiles x 4 groups
        assert r["chunk"] in (1024, 1536, 2048) and r["lambda_tile"] in (16, K) and r["lambda_group"] in (1, 2, 4, 8)
        assert r["n_tried"] == 24 and r["ms"] > 0
        assert ctx.info()["chunk"] == r["chunk"]
        got = ctx.loglik(lt)
        plain = ctx.loglik_plain(lt[:2], grad=False)
        torch.cuda.synchronize()
    def diff(a, b):   # equal finite patterns (a flagged Lambda gives -inf), then the gap
        a = a.cpu().numpy()
        assert np.array_equal(np.isfinite(a), np.isfinite(b))
        f = np.isfinite(b)
        return np.abs(a[f] - b[f]).max() if f.any() else 0.0

    d_ev = diff(got["lnL_event"], ref["lnL_event"])
    d_tot = diff(got["lnL_total"], ref["lnL_total"])
    d_pl = diff(plain["lnL_total"], ref["lnL_total"][:2])
    print(f"autotune {r}: per-event {d_ev:.2e}, total {d_tot:.2e}, plain {d_pl:.2e}")
    assert d_ev <= 1e-5 and d_tot <= 1e-3 and d_pl <= 1e-3
