"""FP64 CPU oracle for the dark-siren hierarchical log-likelihood (test infrastructure).

This package is the independent reference that the CUDA library is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library never does.  The arithmetic lives in
``gwc_oracle.cpp`` (plain C++17, FP64, libm, OpenMP over events); this module only
compiles it with g++ and marshals numpy arrays through ctypes.

Every function is pinned by the tests in ``tests/test_oracle_*.py`` (closed forms,
unit normalisations, invariants, finite differences and a brute-force mpmath
restatement); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

NP = 13       # hyperparameters of the power law + peak mass model
NP_MP = 16    # of the multi-peak model: [..., mu_high, sigma_high, lambda_low]
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwc_oracle.cpp")
_LIB = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liborc.so`` (g++, -O2, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-Wno-unused-function", _SRC, "-o", _LIB + ".tmp"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Inputs(ctypes.Structure):
    _fields_ = [
        ("n_events", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("offsets", ctypes.c_void_p),
        ("m1", ctypes.c_void_p), ("m2", ctypes.c_void_p), ("dl", ctypes.c_void_p),
        ("lnpe", ctypes.c_void_p), ("pix", ctypes.c_void_p),
        ("n_pix", ctypes.c_int32), ("n_z", ctypes.c_int32), ("z_max", ctypes.c_double),
        ("los", ctypes.c_void_p),
        ("n_inj", ctypes.c_int64), ("n_draw", ctypes.c_double),
        ("im1", ctypes.c_void_p), ("im2", ctypes.c_void_p), ("idl", ctypes.c_void_p),
        ("ilnpd", ctypes.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d, i32, i64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            L = _lib
            L.orc_loglik.restype = ctypes.c_int
            L.orc_loglik.argtypes = [ctypes.POINTER(Inputs), i32, vp, i32, i32, d, d, i32,
                                     vp, vp, vp, vp, vp, vp, vp, vp, vp]
            for name, args in [("orc_E", [d, d]), ("orc_I", [d, d]), ("orc_D", [d, d]),
                               ("orc_Dprime", [d, d]), ("orc_z_of_x", [d, d, d]),
                               ("orc_S", [d, d, d]), ("orc_ln_p_m1", [d, vp, i32]),
                               ("orc_ln_p_m2", [d, d, vp, i32]), ("orc_C", [d, vp, i32]),
                               ("orc_ln_Zm1", [vp, i32]), ("orc_ln_psi", [d, vp, i32]),
                               ("orc_ln_Nz", [vp, i32, vp, i32, d]), ("orc_rule_poly", [i32, i32])]:
                fn = getattr(L, name)
                fn.restype = d
                fn.argtypes = args
            L.orc_los_cell.restype = i32
            L.orc_los_cell.argtypes = [ctypes.c_float, i32, d]
            L.orc_sample_cells.restype = ctypes.c_int
            L.orc_sample_cells.argtypes = [vp, i32, i64, vp, i32, d, vp, vp]
            L.orc_ln_w_samples.restype = ctypes.c_int
            L.orc_ln_w_samples.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, vp, i32, i32, d, vp, vp, vp]
            L.orc_ln_w_row.restype = ctypes.c_int
            L.orc_ln_w_row.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, i32, d, vp, vp]
            L.orc_loglik_kde.restype = ctypes.c_int
            L.orc_loglik_kde.argtypes = [ctypes.POINTER(Inputs), i32, vp, i32, i32, i32, d, d, i32,
                                         vp, vp, vp, vp, vp, vp]
            L.orc_num_params.restype = i32
            L.orc_num_params.argtypes = [i32]
            L.orc_bandwidth.restype = d
            L.orc_bandwidth.argtypes = [vp, i64, i32]
        return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _lam(lam):
    """Lambda as float64; its width selects the mass model (13: power law + peak,
    16: multi-peak)."""
    a = np.ascontiguousarray(lam, dtype=np.float64)
    assert a.shape[-1] in (NP, NP_MP), "Lambda rows have 13 or 16 entries"
    return a


def E(z, om): return lib().orc_E(z, om)
def I(z, om): return lib().orc_I(z, om)
def D(z, om): return lib().orc_D(z, om)
def Dprime(z, om): return lib().orc_Dprime(z, om)
def z_of_x(x, om, zmax=10.0): return lib().orc_z_of_x(x, om, zmax)
def S(m, mmin, dm): return lib().orc_S(m, mmin, dm)
def ln_p_m1(m1, lam): a = _lam(lam); return lib().orc_ln_p_m1(m1, _ptr(a), a.shape[-1])
def ln_p_m2(m2, m1, lam): a = _lam(lam); return lib().orc_ln_p_m2(m2, m1, _ptr(a), a.shape[-1])
def C(m1, lam): a = _lam(lam); return lib().orc_C(m1, _ptr(a), a.shape[-1])
def ln_Zm1(lam): a = _lam(lam); return lib().orc_ln_Zm1(_ptr(a), a.shape[-1])
def ln_psi(z, lam): a = _lam(lam); return lib().orc_ln_psi(z, _ptr(a), a.shape[-1])
def rule_poly(k, which): return lib().orc_rule_poly(k, which)


def ln_Nz(lam, pbar, zmax):
    a = _lam(lam)
    p = np.ascontiguousarray(pbar, dtype=np.float64)
    return lib().orc_ln_Nz(_ptr(a), a.shape[-1], _ptr(p), len(p), zmax)


def los_cell(z, nz, zmax):
    """LOS grid cell of the float32 value z (-1 outside [0, zmax])."""
    return lib().orc_los_cell(ctypes.c_float(float(np.float32(z))), nz, zmax)


def sample_cells(lam, dl, nz, zmax):
    """LOS grid cell (int32, -1 where d_L maps outside [0, zmax]) and exact grid position
    z (nz - 1) / zmax (NaN there) of each sample's redshift at Lambda, as ln_w uses them."""
    a = _lam(lam)
    dl = np.ascontiguousarray(dl, dtype=np.float32)
    cell = np.empty(len(dl), np.int32)
    pos = np.empty(len(dl), np.float64)
    if lib().orc_sample_cells(_ptr(a), a.shape[-1], len(dl), _ptr(dl), nz, zmax, _ptr(cell), _ptr(pos)) != 0:
        raise ValueError("Lambda outside its domain")
    return cell, pos


def ln_w_row(lam, m1, m2, dl, lnpi, row, zmax, grad=False):
    """Per-sample ln w against one LOS row (which also defines N_z); -inf where w = 0."""
    a = _lam(lam)
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    m1, m2, dl, lnpi, row = f32(m1), f32(m2), f32(dl), f32(lnpi), f32(row)
    n = len(m1)
    out = np.empty(n, np.float64)
    g = np.empty((n, a.shape[-1]), np.float64) if grad else None
    rc = lib().orc_ln_w_row(_ptr(a), a.shape[-1], n, _ptr(m1), _ptr(m2), _ptr(dl), _ptr(lnpi), _ptr(row),
                            len(row), zmax, _ptr(out), _ptr(g))
    if rc != 0:
        raise ValueError("Lambda outside its domain")
    return (out, g) if grad else out


def ln_w_samples(lam, cat, which="events", idx=None, grad=False):
    """Per-sample ln w exactly as the likelihood uses it: event samples against their
    pixel's LOS row, injections against the pixel mean, N_z from the pixel mean."""
    a = _lam(lam)
    f32 = lambda x: np.ascontiguousarray(x, dtype=np.float32)
    keys = ("m1", "m2", "dl", "lnpe") if which == "events" else ("inj_m1", "inj_m2", "inj_dl", "inj_lnpd")
    sel = slice(None) if idx is None else idx
    m1, m2, dl, lp = (f32(cat[k][sel]) for k in keys)
    pix = np.ascontiguousarray(cat["pix"][sel], dtype=np.int32) if which == "events" else None
    los = f32(cat["los"])
    n = len(m1)
    out = np.empty(n, np.float64)
    g = np.empty((n, a.shape[-1]), np.float64) if grad else None
    kink = np.empty((n, a.shape[-1]), np.float64) if grad else None
    rc = lib().orc_ln_w_samples(_ptr(a), a.shape[-1], n, _ptr(m1), _ptr(m2), _ptr(dl), _ptr(lp),
                                _ptr(pix) if pix is not None else None, _ptr(los), los.shape[0],
                                los.shape[1], float(cat["z_max"]), _ptr(out), _ptr(g),
                                _ptr(kink) if grad else None)
    if rc != 0:
        raise ValueError("Lambda outside its domain")
    return (out, g, kink) if grad else out


BW_RULES = {"scott": 0, "silverman": 1, "biweight": 2}


def bandwidth(z, rule="scott"):
    """KDE bandwidth of the values z by the named rule (see bandwidth() in the C++)."""
    a = np.ascontiguousarray(z, dtype=np.float64)
    return lib().orc_bandwidth(_ptr(a), len(a), BW_RULES[rule])


def _inputs(cat, keep):
    def arr(key, dt):
        a = np.ascontiguousarray(cat[key], dtype=dt)
        keep[key] = a
        return _ptr(a)

    los = np.ascontiguousarray(cat["los"], dtype=np.float32)
    keep["los"] = los
    n_ev = len(cat["offsets"]) - 1
    return n_ev, Inputs(n_events=n_ev, pad0=0, offsets=arr("offsets", np.int64),
                        m1=arr("m1", np.float32), m2=arr("m2", np.float32), dl=arr("dl", np.float32),
                        lnpe=arr("lnpe", np.float32), pix=arr("pix", np.int32),
                        n_pix=los.shape[0], n_z=los.shape[1], z_max=float(cat["z_max"]),
                        los=_ptr(los), n_inj=len(cat["inj_m1"]), n_draw=float(cat["n_draw"]),
                        im1=arr("inj_m1", np.float32), im2=arr("inj_m2", np.float32),
                        idl=arr("inj_dl", np.float32), ilnpd=arr("inj_lnpd", np.float32))


def loglik_kde(cat, lam, bw="scott", n_grid=256, neff_min_pixel=2.0, neff_min_sel=0.0, n_threads=0):
    """The KDE form of the likelihood (Eqs. 5-7): per-pixel weighted Gaussian KDE in z on
    an n_grid-point grid over [0, z_max], times the pixel's LOS prior, trapezoid rule,
    pixels below neff_min_pixel dropped.  neff_event is the effective number of kept
    pixels.  Value only."""
    lam = np.atleast_2d(_lam(lam))
    K = lam.shape[0]
    keep = {}
    n_ev, inp = _inputs(cat, keep)
    out = dict(lnL_event=np.empty((K, n_ev)), neff_event=np.empty((K, n_ev)),
               ln_xi=np.empty(K), neff_sel=np.empty(K), lnL_total=np.empty(K),
               flags=np.empty(K, np.int32))
    rc = lib().orc_loglik_kde(ctypes.byref(inp), K, _ptr(lam), lam.shape[1], BW_RULES[bw], n_grid, neff_min_pixel,
                              neff_min_sel, n_threads, _ptr(out["lnL_event"]), _ptr(out["neff_event"]),
                              _ptr(out["ln_xi"]), _ptr(out["neff_sel"]), _ptr(out["lnL_total"]),
                              _ptr(out["flags"]))
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    return out


def loglik(cat, lam, grad=False, neff_min_event=2.0, neff_min_sel=0.0, n_threads=0):
    """Evaluate the whole likelihood for a Lambda batch ``lam`` [K, 13] (power law +
    peak) or [K, 16] (multi-peak); gradients have the same width.

    ``cat`` is a dict of numpy arrays with the keys produced by
    ``paper_2605_23538_gb300.synth`` (offsets, m1, m2, dl, lnpe, pix, los, z_max,
    inj_m1, inj_m2, inj_dl, inj_lnpd, n_draw).  Returns a dict of outputs.
    """
    lam = np.atleast_2d(_lam(lam))
    K = lam.shape[0]
    keep = {}

    def arr(key, dt):
        a = np.ascontiguousarray(cat[key], dtype=dt)
        keep[key] = a
        return _ptr(a)

    los = np.ascontiguousarray(cat["los"], dtype=np.float32)
    keep["los"] = los
    n_ev = len(cat["offsets"]) - 1
    inp = Inputs(n_events=n_ev, pad0=0, offsets=arr("offsets", np.int64),
                 m1=arr("m1", np.float32), m2=arr("m2", np.float32), dl=arr("dl", np.float32),
                 lnpe=arr("lnpe", np.float32), pix=arr("pix", np.int32),
                 n_pix=los.shape[0], n_z=los.shape[1], z_max=float(cat["z_max"]),
                 los=_ptr(los), n_inj=len(cat["inj_m1"]), n_draw=float(cat["n_draw"]),
                 im1=arr("inj_m1", np.float32), im2=arr("inj_m2", np.float32),
                 idl=arr("inj_dl", np.float32), ilnpd=arr("inj_lnpd", np.float32))
    P = lam.shape[1]
    out = dict(lnL_event=np.empty((K, n_ev)), neff_event=np.empty((K, n_ev)),
               ln_xi=np.empty(K), neff_sel=np.empty(K), lnL_total=np.empty(K),
               flags=np.empty(K, np.int32), grad_total=np.zeros((K, P)) if grad else None,
               grad_scale=np.zeros((K, P)) if grad else None,
               grad_kink=np.zeros((K, P)) if grad else None)
    rc = lib().orc_loglik(ctypes.byref(inp), K, _ptr(lam), P, int(bool(grad)), neff_min_event,
                          neff_min_sel, n_threads, _ptr(out["lnL_event"]), _ptr(out["neff_event"]),
                          _ptr(out["ln_xi"]), _ptr(out["neff_sel"]), _ptr(out["lnL_total"]),
                          _ptr(out["flags"]), _ptr(out["grad_total"]), _ptr(out["grad_scale"]),
                          _ptr(out["grad_kink"]))
    if rc != 0:
        raise ValueError("oracle rejected the inputs")
    if not grad:
        del out["grad_total"], out["grad_scale"], out["grad_kink"]
    return out
