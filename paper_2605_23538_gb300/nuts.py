"""Multi-walker No-U-Turn sampler over the library's batched log-likelihood and gradient.

The sampler is the efficient No-U-Turn Sampler of Hoffman & Gelman (2014, JMLR 15, their
Algorithm 3, with the dual-averaging step-size adaptation of their Algorithm 6): a slice
variable, trees doubled in a random direction until a U-turn or a divergence, and a
uniform choice among the tree's points that lie in the slice.  Here it runs K walkers
(independent chains) at once, each with its own tree, its own random stream and its own
step size, and with a diagonal mass matrix: kinetic energy p.M^-1.p / 2, and the U-turn
test on the velocities M^-1 p.

Each walker's tree building is a generator that yields the point it needs next and
receives (log-likelihood, gradient) there; the driver collects the pending points of all
walkers and evaluates them in one batched call (one gwc_loglik_grad launch on the GPU), so
walkers with trees of different depths still share every evaluation.  A walker's chain
depends only on its seed, not on which other walkers share its batches.

The target is any callable logp_grad(q [n, P]) -> (lnL [n], grad [n, P]); Context.loglik_grad
gives one with `context_target`.  A point where lnL is -inf (outside the Lambda domain, or
flagged) ends the subtree that reaches it.
"""
from __future__ import annotations

import numpy as np

DELTA_MAX = 1000.0   # energy error beyond which a trajectory counts as divergent


class _State:
    """A phase-space point with its log-likelihood and gradient."""
    __slots__ = ("q", "p", "lnL", "grad")

    def __init__(self, q, p, lnL, grad):
        self.q, self.p, self.lnL, self.grad = q, p, lnL, grad


class _Walker:
    def __init__(self, q, lnL, grad, eps, inv_mass, seed, max_depth):
        self.q, self.lnL, self.grad = q, lnL, grad
        self.eps = eps
        self.inv_mass = inv_mass
        self.rng = np.random.default_rng(seed)
        self.max_depth = max_depth

    def kinetic(self, p):
        return 0.5 * float(np.dot(self.inv_mass * p, p))

    def leapfrog(self, s, step):
        """One leapfrog step of signed size `step` from state s (a generator: it yields the
        new position and receives its (lnL, grad))."""
        p_half = s.p + 0.5 * step * s.grad
        q = s.q + step * self.inv_mass * p_half
        lnL, grad = yield q
        grad = np.asarray(grad, dtype=np.float64)
        if not np.isfinite(lnL) or not np.all(np.isfinite(grad)):
            return _State(q, p_half, -np.inf, np.zeros_like(grad))
        return _State(q, p_half + 0.5 * step * grad, float(lnL), grad)

    def no_uturn(self, minus, plus):
        dq = plus.q - minus.q
        return np.dot(dq, self.inv_mass * minus.p) >= 0.0 and np.dot(dq, self.inv_mass * plus.p) >= 0.0

    def build_tree(self, s, log_u, v, j, H0):
        """Subtree of 2^j leapfrog steps in direction v from s.  Returns (minus, plus,
        proposal, n in slice, continue, sum of acceptance statistics, their count)."""
        if j == 0:
            s1 = yield from self.leapfrog(s, v * self.eps)
            H1 = -s1.lnL + self.kinetic(s1.p) if np.isfinite(s1.lnL) else np.inf
            n = 1 if log_u <= -H1 else 0
            ok = log_u < DELTA_MAX - H1
            alpha = min(1.0, np.exp(H0 - H1)) if np.isfinite(H1) else 0.0
            return s1, s1, s1, n, ok, alpha, 1
        minus, plus, prop, n, ok, a, na = yield from self.build_tree(s, log_u, v, j - 1, H0)
        if ok:
            if v < 0:
                minus, _, prop2, n2, ok2, a2, na2 = yield from self.build_tree(minus, log_u, v, j - 1, H0)
            else:
                _, plus, prop2, n2, ok2, a2, na2 = yield from self.build_tree(plus, log_u, v, j - 1, H0)
            if n + n2 > 0 and self.rng.random() < n2 / (n + n2):
                prop = prop2
            a, na = a + a2, na + na2
            n += n2
            ok = ok2 and self.no_uturn(minus, plus)
        return minus, plus, prop, n, ok, a, na

    def iterate(self):
        """One NUTS transition (a generator over the walker's evaluation requests);
        returns (tree depth, leapfrog steps, mean acceptance statistic)."""
        p0 = self.rng.standard_normal(self.q.shape) / np.sqrt(self.inv_mass)
        s0 = _State(self.q, p0, self.lnL, self.grad)
        H0 = -self.lnL + self.kinetic(p0)
        log_u = -H0 + np.log(self.rng.random())   # the slice: u ~ U(0, exp(-H0))
        minus = plus = prop = s0
        n, ok, j, a, na = 1, True, 0, 0.0, 0
        while ok and j < self.max_depth:
            v = 1 if self.rng.random() < 0.5 else -1
            if v < 0:
                minus, _, prop2, n2, ok2, a2, na2 = yield from self.build_tree(minus, log_u, v, j, H0)
            else:
                _, plus, prop2, n2, ok2, a2, na2 = yield from self.build_tree(plus, log_u, v, j, H0)
            if ok2 and self.rng.random() < min(1.0, n2 / n):
                prop = prop2
            n += n2
            a, na = a + a2, na + na2
            ok = ok2 and self.no_uturn(minus, plus)
            j += 1
        self.q, self.lnL, self.grad = prop.q, prop.lnL, prop.grad
        return j, na, a / max(na, 1)


def sample(logp_grad, q0, n_samples, eps, inv_mass=None, seed=0, n_adapt=0, target_accept=0.8,
           max_depth=10):
    """Run K walkers from the rows of q0 [K, P]: n_adapt transitions that adapt each walker's
    step size by dual averaging (discarded), then n_samples recorded transitions.

    eps: initial step size (scalar or [K]); inv_mass: diagonal of M^-1 ([P], default ones).
    Returns a dict: samples [n_samples, K, P], lnL [n_samples, K], depth and n_leapfrog
    [n_samples, K], accept_stat [n_samples, K], eps [K] (the step sizes used for the
    recorded transitions), n_calls (batched evaluations made in all) and calls
    [n_samples] (those of each recorded transition: every call serves each walker still
    building its tree, so a transition takes as many calls as its longest walker takes
    leapfrog steps)."""
    q0 = np.atleast_2d(np.asarray(q0, dtype=np.float64))
    K, P = q0.shape
    inv_mass = np.ones(P) if inv_mass is None else np.asarray(inv_mass, dtype=np.float64).reshape(P)
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (K,)).copy()
    lnL, grad = logp_grad(q0)
    lnL, grad = np.asarray(lnL, dtype=np.float64), np.asarray(grad, dtype=np.float64)
    if not np.all(np.isfinite(lnL)):
        raise ValueError("every starting point needs a finite log-likelihood")
    walkers = [_Walker(q0[k].copy(), float(lnL[k]), grad[k].copy(), eps[k], inv_mass,
                       np.random.SeedSequence([seed, k]), max_depth) for k in range(K)]
    # dual averaging (Hoffman & Gelman's Algorithm 6 constants)
    gamma, t0, kappa = 0.05, 10.0, 0.75
    mu = np.log(10.0 * eps)
    hbar = np.zeros(K)
    log_eps_bar = np.zeros(K)
    out = dict(samples=np.empty((n_samples, K, P)), lnL=np.empty((n_samples, K)),
               depth=np.empty((n_samples, K), np.int32), n_leapfrog=np.empty((n_samples, K), np.int32),
               accept_stat=np.empty((n_samples, K)), calls=np.empty(n_samples, np.int64))
    n_calls = 1
    for it in range(n_adapt + n_samples):
        gens = [w.iterate() for w in walkers]
        pending = {k: next(g) for k, g in enumerate(gens)}   # every transition takes a step
        results = {}
        calls_before = n_calls
        while pending:
            ks = sorted(pending)
            L, G = logp_grad(np.stack([pending[k] for k in ks]))
            n_calls += 1
            for i, k in enumerate(ks):
                try:
                    pending[k] = gens[k].send((L[i], G[i]))
                except StopIteration as stop:
                    results[k] = stop.value
                    del pending[k]
        if it < n_adapt:
            m = it + 1
            for k, w in enumerate(walkers):
                alpha = results[k][2]
                hbar[k] = (1.0 - 1.0 / (m + t0)) * hbar[k] + (target_accept - alpha) / (m + t0)
                log_eps = mu[k] - np.sqrt(m) / gamma * hbar[k]
                w.eps = float(np.exp(log_eps))
                log_eps_bar[k] = m ** -kappa * log_eps + (1.0 - m ** -kappa) * log_eps_bar[k]
            if it == n_adapt - 1:
                for k, w in enumerate(walkers):
                    w.eps = float(np.exp(log_eps_bar[k]))
            continue
        r = it - n_adapt
        out["calls"][r] = n_calls - calls_before
        for k, w in enumerate(walkers):
            out["samples"][r, k] = w.q
            out["lnL"][r, k] = w.lnL
            out["depth"][r, k], out["n_leapfrog"][r, k], out["accept_stat"][r, k] = results[k]
    out["eps"] = np.array([w.eps for w in walkers])
    out["n_calls"] = n_calls
    return out


def context_target(context, device="cuda"):
    """logp_grad over a Context: one gwc_loglik_grad call per batch of points (at most the
    context's max_K of them), totals and gradients copied to the host."""
    import torch

    def logp_grad(q):
        lam = torch.as_tensor(np.ascontiguousarray(q), dtype=torch.float64, device=device)
        r = context.loglik_grad(lam)
        return r["lnL_total"].cpu().numpy(), r["grad_total"].cpu().numpy()

    return logp_grad
