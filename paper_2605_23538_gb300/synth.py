"""Seeded synthetic inputs with the shapes of the paper's workloads.

The paper's inputs (mock O5 parameter-estimation samples, GWTC-4 samples, GLADE+
line-of-sight priors, the LVK injection set) are not available, so catalogues are
drawn here from fixed seeds with the sizes, value distributions and structure of the
workloads the paper describes (Sec. 3.1, App. A): ragged events whose samples sit in
a block of neighbouring HEALPix pixels, LOS redshift priors on a uniform z grid that
mix a smooth volume term with narrow galaxy peaks, and a detected-injection set with
a known draw density.

This module deliberately holds none of the likelihood's arithmetic.  Sources are
placed with an analytic fit to the flat-LCDM luminosity distance (U.-L. Pen 1999,
ApJS 120, 49) rather than the quadrature the likelihood uses, and masses are drawn
from closed-form inverse CDFs of a power law and a Gaussian, without the smoothing
window or any normalisation integral.  Both the CUDA library and the oracle consume
these arrays as opaque inputs.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

SEED_BASE = 20260523
C_KMS = 299792.458

# Lambda = [H0, Om, alpha, beta, m_min, m_max, delta_m, mu_g, sigma_g, lambda_peak,
#           gamma, kappa, z_p]; the values at which the synthetic sources are drawn.
LAMBDA_NAMES = ("H0", "Om", "alpha", "beta", "m_min", "m_max", "delta_m", "mu_g",
                "sigma_g", "lambda_peak", "gamma", "kappa", "z_p")
FIDUCIAL = np.array([70.0, 0.3, 3.4, 1.1, 5.0, 90.0, 4.0, 34.0, 4.0, 0.04, 2.7, 3.0, 2.0])

# The multi-peak mass model takes 16: the first Gaussian is the lower-mass peak, and
# three more entries give the higher-mass peak and the low peak's share of lambda_g.
# Its reference point is the paper's Table 2 (the injected values of its simulated O5
# catalogue).
LAMBDA_NAMES_MP = LAMBDA_NAMES[:7] + ("mu_low", "sigma_low", "lambda_g") + LAMBDA_NAMES[10:] + \
    ("mu_high", "sigma_high", "lambda_low")
FIDUCIAL_MP = np.array([67.4, 0.315, 2.9, 1.0, 4.6, 86.3, 4.8, 9.7, 0.7, 0.4, 3.3, 2.9, 2.5,
                        30.7, 6.3, 0.8])

_D0_MPC = 8000.0      # SNR normalisation distance of the toy detector
_SNR_THRESHOLD = 12.0
_INJ_DLMAX = 20000.0  # injections: p(dL) = 2 dL / dLmax^2 on (0, dLmax]
_INJ_M_LO, _INJ_M_HI = 2.0, 500.0


@dataclass(frozen=True)
class Workload:
    name: str
    n_events: int
    samples: tuple          # ("fixed", n) | ("uniform", lo, hi) | ("loguniform", lo, hi)
    nside: int
    n_z: int
    n_inj: int              # stored (detected) injections; for "draws" mode, draws
    inj_mode: str           # "found" or "draws"
    K: int
    z_max: float = 2.0

    @property
    def n_pix(self) -> int:
        return 12 * self.nside * self.nside


WORKLOADS = {
    # plain method, tiny: 10 events x 1000 samples, nside 8 x 512 z, 1e4 injections drawn
    "c1": Workload("c1", 10, ("fixed", 1000), 8, 512, 10_000, "draws", 1),
    # current-catalogue scale: 150 events x U{2000..8000}, nside 32 x 2048 z, 1e6 injections
    "c2": Workload("c2", 150, ("uniform", 2000, 8000), 32, 2048, 1_000_000, "found", 64),
    # O5-like: 2000 events, log-uniform 1k..16k samples, nside 64 x 2048 z, 1e7 injections
    "c3": Workload("c3", 2000, ("loguniform", 1000, 16000), 64, 2048, 10_000_000, "found", 256),
    # precision and scale stress: 10000 events x 4096, 5e7 injections
    "c5": Workload("c5", 10_000, ("fixed", 4096), 64, 2048, 50_000_000, "found", 128),
}


def rng(purpose: int, seed: int = SEED_BASE) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, purpose])))


def dl_fit(z, H0=70.0, om=0.3):
    """Pen (1999) analytic fit to the flat-LCDM luminosity distance [Mpc]."""
    z = np.asarray(z, dtype=np.float64)
    s = ((1.0 - om) / om) ** (1.0 / 3.0)

    def eta(a):
        return 2.0 * math.sqrt(s ** 3 + 1.0) * (
            1.0 / a ** 4 - 0.1540 * s / a ** 3 + 0.4304 * s ** 2 / a ** 2
            + 0.19097 * s ** 3 / a + 0.066941 * s ** 4) ** (-0.125)

    return (C_KMS / H0) * (1.0 + z) * (eta(1.0) - eta(1.0 / (1.0 + z)))


def _trap_weights(n, dz):
    w = np.full(n, dz)
    w[0] = w[-1] = 0.5 * dz
    return w


def los_table(n_pix: int, n_z: int, z_max: float = 2.0, n_gal: int = 50, seed: int = SEED_BASE,
              chunk: int = 1024, workers: int | None = None) -> np.ndarray:
    """[n_pix, n_z] float32 LOS redshift priors on z_j = j z_max / (n_z - 1).

    Each row is 0.5 x (uniform in comoving volume) + 0.5 x (mean of n_gal Gaussian
    galaxies, sigma = 0.003 (1 + z_g), centres drawn from the volume law, each cut at
    5 sigma and normalised on the grid), and the row is normalised to unit trapezoid
    area.  All random numbers are drawn up front, so the result does not depend on
    how the pixel chunks are scheduled over threads.
    """
    from concurrent.futures import ThreadPoolExecutor

    g = rng(1, seed)
    z = np.linspace(0.0, z_max, n_z)
    dz = z[1] - z[0]
    tw = _trap_weights(n_z, dz)
    dc = dl_fit(np.maximum(z, 1e-9)) / (1.0 + z)
    vol = dc ** 2 * np.gradient(dc, z)
    vol[0] = 0.0
    vol /= np.sum(vol * tw)
    cdf = np.cumsum(vol * tw)
    cdf /= cdf[-1]
    zg_all = np.interp(g.random((n_pix, n_gal)), cdf, z)
    out = np.empty((n_pix, n_z), dtype=np.float32)
    half = int(math.ceil(5.0 * 0.003 * (1.0 + z_max) / dz)) + 1
    offs = np.arange(-half, half + 1, dtype=np.float32)
    vol32 = vol.astype(np.float32)
    tw32 = tw.astype(np.float32)

    def work(p0):
        p1 = min(n_pix, p0 + chunk)
        npc = p1 - p0
        zg = zg_all[p0:p1].astype(np.float32)
        inv_s = (1.0 / (0.003 * (1.0 + zg))).astype(np.float32)
        j0 = np.rint(zg / dz).astype(np.int64)
        idx = j0[:, :, None] + offs.astype(np.int64)[None, None, :]
        x = ((j0[:, :, None] + offs[None, None, :]) * np.float32(dz) - zg[:, :, None]) * inv_s[:, :, None]
        val = np.exp(np.float32(-0.5) * x * x)
        val[(idx < 0) | (idx >= n_z)] = 0.0
        np.clip(idx, 0, n_z - 1, out=idx)
        norm = np.sum(val * tw32[idx], axis=2, keepdims=True)
        val /= np.maximum(norm, np.float32(1e-30)) * np.float32(n_gal)
        flat = (np.arange(npc)[:, None, None] * n_z + idx).ravel()
        gal = np.bincount(flat, weights=val.ravel(), minlength=npc * n_z).reshape(npc, n_z)
        row = 0.5 * vol32[None, :] + 0.5 * gal
        row /= np.sum(row * tw[None, :], axis=1, keepdims=True)
        out[p0:p1] = row.astype(np.float32)

    nw = workers or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(nw) as ex:
        list(ex.map(work, range(0, n_pix, chunk)))
    return out


def _chirp_mass(m1, m2):
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def _detected(g, m1d, m2d, dl):
    omega = g.random(len(m1d))
    snr = 8.0 * (_chirp_mass(m1d, m2d) / 10.0) ** (5.0 / 6.0) * (_D0_MPC / dl) * omega
    return snr > _SNR_THRESHOLD


def _sample_counts(w: Workload, g) -> np.ndarray:
    kind = w.samples[0]
    if kind == "fixed":
        return np.full(w.n_events, int(w.samples[1]), dtype=np.int64)
    if kind == "uniform":
        return g.integers(int(w.samples[1]), int(w.samples[2]) + 1, size=w.n_events).astype(np.int64)
    if kind == "loguniform":
        lo, hi = math.log(w.samples[1]), math.log(w.samples[2])
        return np.rint(np.exp(g.uniform(lo, hi, size=w.n_events))).astype(np.int64)
    raise ValueError(kind)


def _source_truths(n, los, z_max, g):
    """n detected sources: pixel block, z, detector-frame masses and distance."""
    n_pix, n_z = los.shape
    z = np.linspace(0.0, z_max, n_z)
    block = min(20, n_pix)
    out = {k: [] for k in ("start", "pix", "z", "m1d", "m2d", "dl")}
    have = 0
    while have < n:
        m = max(4 * (n - have), 256)
        start = g.integers(0, n_pix - block + 1, size=m)
        pix = start + g.integers(0, block, size=m)
        # z from the pixel's LOS prior times a (1+z)^1.7 rate, by inverse CDF on the grid
        dens = los[pix].astype(np.float64) * (1.0 + z[None, :]) ** 1.7
        cdf = np.cumsum(dens, axis=1)
        cdf /= cdf[:, -1:]
        u = g.random(m)
        j = np.minimum((cdf < u[:, None]).sum(axis=1), n_z - 1)
        zs = np.clip(z[j] - g.random(m) * (z[1] - z[0]), 1e-3, z_max)
        # masses: power law (alpha = 3.4) on [5, 90] or, with probability 0.04, N(34, 4)
        a = 1.0 - 3.4
        lo, hi = 5.0 ** a, 90.0 ** a
        m1 = (lo + g.random(m) * (hi - lo)) ** (1.0 / a)
        peak = g.random(m) < 0.04
        m1[peak] = np.clip(g.normal(34.0, 4.0, size=int(peak.sum())), 5.0, 90.0)
        b = 1.0 + 1.1
        m2 = (5.0 ** b + g.random(m) * (m1 ** b - 5.0 ** b)) ** (1.0 / b)
        dl = dl_fit(zs)
        m1d, m2d = m1 * (1.0 + zs), m2 * (1.0 + zs)
        keep = _detected(g, m1d, m2d, dl)
        for k, v in (("start", start), ("pix", pix), ("z", zs), ("m1d", m1d), ("m2d", m2d), ("dl", dl)):
            out[k].append(v[keep])
        have += int(keep.sum())
    return {k: np.concatenate(v)[:n] for k, v in out.items()}


def events(w: Workload, los: np.ndarray, seed: int = SEED_BASE) -> dict:
    """Posterior samples for w.n_events detected sources, CSR by event, sorted by pixel."""
    g = rng(2, seed)
    n_pix = los.shape[0]
    block = min(20, n_pix)
    tr = _source_truths(w.n_events, los, w.z_max, g)
    counts = _sample_counts(w, g)
    offsets = np.zeros(w.n_events + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    ns = int(offsets[-1])
    ev = np.repeat(np.arange(w.n_events), counts)
    dl = tr["dl"][ev] * (1.0 + 0.3 * g.standard_normal(ns))
    bad = dl <= 0.0
    while bad.any():  # truncate to dL > 0 by redrawing
        dl[bad] = tr["dl"][ev[bad]] * (1.0 + 0.3 * g.standard_normal(int(bad.sum())))
        bad = dl <= 0.0
    m1 = tr["m1d"][ev] * (1.0 + 0.1 * g.standard_normal(ns))
    m2 = tr["m2d"][ev] * (1.0 + 0.1 * g.standard_normal(ns))
    m1, m2 = np.maximum(m1, m2), np.minimum(m1, m2)
    pix = tr["start"][ev] + g.integers(0, block, size=ns)
    order = np.lexsort((pix, ev))
    cat = dict(offsets=offsets, m1=m1[order].astype(np.float32), m2=m2[order].astype(np.float32),
               dl=dl[order].astype(np.float32), pix=pix[order].astype(np.int32))
    cat["lnpe"] = (2.0 * np.log(cat["dl"].astype(np.float64))).astype(np.float32)
    return cat


def injections(w: Workload, seed: int = SEED_BASE, chunk: int = 1 << 22) -> dict:
    """Detected injections with their analytic draw density.

    Draws: ln m1d ~ U(ln 2, ln 500); m2d | m1d ~ U(2, m1d); p(dL) = 2 dL / dLmax^2 on
    (0, dLmax].  Detection: the toy-detector SNR above 12.  In "draws" mode a fixed
    number of draws is made and the detected subset stored; in "found" mode draws
    continue until w.n_inj are detected, and n_draw counts every draw made up to the
    last one kept.
    """
    g = rng(3, seed)
    keep = {k: [] for k in ("m1", "m2", "dl")}
    n_found, n_draw = 0, 0
    target = w.n_inj
    lnr = math.log(_INJ_M_HI / _INJ_M_LO)
    while True:
        m = chunk if w.inj_mode == "found" else min(chunk, target - n_draw)
        if m <= 0:
            break
        m1 = np.exp(math.log(_INJ_M_LO) + lnr * g.random(m))
        m2 = _INJ_M_LO + (m1 - _INJ_M_LO) * g.random(m)
        dl = _INJ_DLMAX * np.sqrt(g.random(m))
        det = _detected(g, m1, m2, dl)
        if w.inj_mode == "found":
            idx = np.flatnonzero(det)
            need = target - n_found
            if len(idx) >= need:
                idx = idx[:need]
                n_draw += int(idx[-1]) + 1 if need > 0 else 0
                n_found += need
                for k, v in (("m1", m1), ("m2", m2), ("dl", dl)):
                    keep[k].append(v[idx])
                break
            n_draw += m
            n_found += len(idx)
        else:
            idx = np.flatnonzero(det)
            n_draw += m
            n_found += len(idx)
        for k, v in (("m1", m1), ("m2", m2), ("dl", dl)):
            keep[k].append(v[idx])
    m1 = np.concatenate(keep["m1"]).astype(np.float32)
    m2 = np.concatenate(keep["m2"]).astype(np.float32)
    dl = np.concatenate(keep["dl"]).astype(np.float32)
    m1d, m2d, dld = (a.astype(np.float64) for a in (m1, m2, dl))
    lnpd = (-np.log(m1d) - math.log(lnr) - np.log(m1d - _INJ_M_LO)
            + math.log(2.0) + np.log(dld) - 2.0 * math.log(_INJ_DLMAX))
    return dict(inj_m1=m1, inj_m2=m2, inj_dl=dl, inj_lnpd=lnpd.astype(np.float32),
                n_draw=float(n_draw))


def lambda_batch(K: int, seed: int = SEED_BASE, purpose: int = 4, model: str = "plp") -> np.ndarray:
    """K Lambda points: H0 ~ U(20, 140), Om ~ U(0.1, 0.5), the rest within +-20% of
    FIDUCIAL (model "plp", 13 columns) or of FIDUCIAL_MP (model "multipeak", 16)."""
    g = rng(purpose, seed)
    fid = FIDUCIAL_MP if model == "multipeak" else FIDUCIAL
    if model not in ("plp", "multipeak"):
        raise ValueError("model is 'plp' or 'multipeak'")
    lam = fid[None, :] * g.uniform(0.8, 1.2, size=(K, len(fid)))
    lam[:, 0] = g.uniform(20.0, 140.0, size=K)
    lam[:, 1] = g.uniform(0.1, 0.5, size=K)
    return lam


def catalogue(w: Workload | str, seed: int = SEED_BASE) -> dict:
    """Everything one likelihood needs: events, LOS table and injections."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    los = los_table(w.n_pix, w.n_z, w.z_max, seed=seed)
    cat = events(w, los, seed=seed)
    cat.update(injections(w, seed=seed))
    cat["los"] = los
    cat["z_max"] = float(w.z_max)
    return cat


def scaled(name: str, n_events: int, samples: tuple, nside: int, n_z: int, n_inj: int,
           inj_mode: str = "found", K: int = 1) -> Workload:
    """A smaller workload with the same recipe (for tests the oracle finishes quickly)."""
    return Workload(name, n_events, samples, nside, n_z, n_inj, inj_mode, K)


def subset_events(cat: dict, idx) -> dict:
    """The same catalogue restricted to the events in ``idx`` (LOS and injections kept)."""
    idx = np.asarray(idx, dtype=np.int64)
    off = cat["offsets"]
    parts = [np.arange(off[i], off[i + 1]) for i in idx]
    sel = np.concatenate(parts) if parts else np.zeros(0, np.int64)
    counts = np.array([len(p) for p in parts], dtype=np.int64)
    out = dict(cat)
    out["offsets"] = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    for k in ("m1", "m2", "dl", "lnpe", "pix"):
        out[k] = cat[k][sel]
    return out
