"""Python binding of libgwc.so, the GB300 dark-siren hierarchical likelihood.

Argument marshalling only: every step of the likelihood runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams; there is no CPU fallback, and
every entry point raises if the compiled library is missing or a call fails.

Names mirror the C ABI in include/gwc.h:
    create / destroy / loglik / loglik_grad / loglik_plain / loglik_grad_host /
    get_info / last_error / los_cell_index / default_options
The ``Context`` class wraps a gwc_ctx, and ``GwcLogLik`` is the autograd.Function
whose backward applies the gradient computed in the same pass as the value.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

NUM_PARAMS = 13               # Lambda entries, power law + peak mass model
NUM_PARAMS_MULTIPEAK = 16     # Lambda entries, multi-peak mass model
MASS_PLP, MASS_MULTIPEAK = 0, 1
MASS_MODELS = {"plp": MASS_PLP, "multipeak": MASS_MULTIPEAK}
FLAG_DOMAIN, FLAG_NEFF_EVENT, FLAG_NEFF_SEL, FLAG_XI_ZERO = 1, 2, 4, 8
LOS_F32, LOS_BF16 = 0, 1
STATUS = {0: "GWC_OK", -1: "GWC_E_INVALID", -2: "GWC_E_CUDA", -3: "GWC_E_NOMEM",
          -4: "GWC_E_TIMEOUT", -5: "GWC_E_UNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgwc.so")
_lock = threading.Lock()
_lib = None


class GwcError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class Events(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int32), ("offsets", ctypes.c_void_p),
                ("m1_det", ctypes.c_void_p), ("m2_det", ctypes.c_void_p),
                ("dl_mpc", ctypes.c_void_p), ("ln_pe_prior", ctypes.c_void_p),
                ("pix", ctypes.c_void_p)]


class Los(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int32), ("n_z", ctypes.c_int32), ("z_max", ctypes.c_double),
                ("dtype", ctypes.c_int32), ("p_z", ctypes.c_void_p)]


class Injections(ctypes.Structure):
    _fields_ = [("n_found", ctypes.c_int64), ("n_draw", ctypes.c_double),
                ("m1_det", ctypes.c_void_p), ("m2_det", ctypes.c_void_p),
                ("dl_mpc", ctypes.c_void_p), ("ln_p_draw", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("neff_min_event", ctypes.c_double), ("neff_min_sel", ctypes.c_double),
                ("accum", ctypes.c_int32), ("los_dtype", ctypes.c_int32),
                ("n_x_table", ctypes.c_int32), ("max_K", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("lambda_tile", ctypes.c_int32),
                ("lambda_group", ctypes.c_int32), ("cap_per_pixel", ctypes.c_int32),
                ("cap_seed", ctypes.c_uint64), ("mass_model", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int32), ("n_samples", ctypes.c_int64),
                ("n_injections", ctypes.c_int64), ("n_pix", ctypes.c_int32),
                ("n_z", ctypes.c_int32), ("n_items", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("n_x_table", ctypes.c_int32), ("max_K", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("n_params", ctypes.c_int32),
                ("mass_model", ctypes.c_int32)]


class KdeOptions(ctypes.Structure):
    _fields_ = [("bw_rule", ctypes.c_int32), ("n_grid", ctypes.c_int32),
                ("neff_min_pixel", ctypes.c_double)]


BW_RULES = {"scott": 0, "silverman": 1, "biweight": 2}


class TuneResult(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("lambda_tile", ctypes.c_int32),
                ("lambda_group", ctypes.c_int32), ("n_tried", ctypes.c_int32),
                ("ms", ctypes.c_double)]


EXPORTS = ("gwc_default_options", "gwc_create", "gwc_loglik", "gwc_loglik_grad",
           "gwc_loglik_plain", "gwc_loglik_grad_host", "gwc_destroy", "gwc_last_error",
           "gwc_get_info", "gwc_los_cell_index", "gwc_profile_enable", "gwc_profile_read",
           "gwc_sample_terms", "gwc_sample_terms_noalloc", "gwc_graph_create", "gwc_graph_launch",
           "gwc_graph_destroy", "gwc_hmc_create", "gwc_hmc_launch", "gwc_hmc_destroy",
           "gwc_autotune", "gwc_default_kde_options", "gwc_loglik_kde", "gwc_loglik_parts",
           "gwc_path_census", "gwc_kde_census", "gwc_alu_probe", "gwc_merge_parts")


def lib():
    """Load libgwc.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2605_23538_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.gwc_default_options.restype = None
        L.gwc_default_options.argtypes = [ctypes.POINTER(Options)]
        L.gwc_create.restype = ctypes.c_int
        L.gwc_create.argtypes = [ctypes.POINTER(Events), ctypes.POINTER(Los),
                                 ctypes.POINTER(Injections), ctypes.POINTER(Options),
                                 ctypes.POINTER(vp)]
        L.gwc_loglik.restype = ctypes.c_int
        L.gwc_loglik.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gwc_loglik_grad.restype = ctypes.c_int
        L.gwc_loglik_grad.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gwc_loglik_plain.restype = ctypes.c_int
        L.gwc_loglik_plain.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gwc_loglik_grad_host.restype = ctypes.c_int
        L.gwc_loglik_grad_host.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.gwc_destroy.restype = None
        L.gwc_destroy.argtypes = [vp]
        L.gwc_last_error.restype = ctypes.c_char_p
        L.gwc_last_error.argtypes = [vp]
        L.gwc_get_info.restype = ctypes.c_int
        L.gwc_get_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.gwc_sample_terms.restype = ctypes.c_int
        L.gwc_sample_terms.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.gwc_sample_terms_noalloc.restype = ctypes.c_int
        L.gwc_sample_terms_noalloc.argtypes = [vp, i64, vp, vp, i64, vp, i32, i32, d, vp, i32,
                                               vp, vp, vp, vp]
        L.gwc_profile_enable.restype = ctypes.c_int
        L.gwc_profile_enable.argtypes = [vp, i32]
        L.gwc_profile_read.restype = ctypes.c_int
        L.gwc_profile_read.argtypes = [vp, vp, vp]
        L.gwc_los_cell_index.restype = ctypes.c_int
        L.gwc_los_cell_index.argtypes = [vp, i64, i32, d, vp, vp]
        L.gwc_graph_create.restype = ctypes.c_int
        L.gwc_graph_create.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp,
                                       ctypes.POINTER(ctypes.c_void_p)]
        L.gwc_graph_launch.restype = ctypes.c_int
        L.gwc_graph_launch.argtypes = [vp, vp]
        L.gwc_graph_destroy.restype = None
        L.gwc_graph_destroy.argtypes = [vp]
        L.gwc_hmc_create.restype = ctypes.c_int
        L.gwc_hmc_create.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                     ctypes.POINTER(ctypes.c_void_p)]
        L.gwc_hmc_launch.restype = ctypes.c_int
        L.gwc_hmc_launch.argtypes = [vp, vp]
        L.gwc_hmc_destroy.restype = None
        L.gwc_hmc_destroy.argtypes = [vp]
        L.gwc_default_kde_options.restype = None
        L.gwc_default_kde_options.argtypes = [ctypes.POINTER(KdeOptions)]
        L.gwc_loglik_kde.restype = ctypes.c_int
        L.gwc_loglik_kde.argtypes = [vp, i32, vp, ctypes.POINTER(KdeOptions), vp, vp, vp, vp, vp, vp, vp]
        L.gwc_loglik_parts.restype = ctypes.c_int
        L.gwc_loglik_parts.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gwc_path_census.restype = ctypes.c_int
        L.gwc_path_census.argtypes = [vp, i32, vp, vp, vp]
        L.gwc_merge_parts.restype = ctypes.c_int
        L.gwc_merge_parts.argtypes = [i32, i32, i32, vp, i32, vp, vp, vp, vp, vp, vp]
        L.gwc_kde_census.restype = ctypes.c_int
        L.gwc_kde_census.argtypes = [vp, i32, vp, ctypes.POINTER(KdeOptions), vp, vp]
        L.gwc_alu_probe.restype = ctypes.c_int
        L.gwc_alu_probe.argtypes = [i32, i32, i32, ctypes.POINTER(d), vp]
        L.gwc_autotune.restype = ctypes.c_int
        L.gwc_autotune.argtypes = [vp, i32, vp, i32, vp, ctypes.POINTER(TuneResult)]
        _lib = L
        return L


def default_options(**kw) -> Options:
    """gwc_default_options with fields overridden by keyword (mass_model may be given by
    name, "plp" or "multipeak")."""
    o = Options()
    lib().gwc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "mass_model" and isinstance(v, str):
            v = MASS_MODELS[v]
        setattr(o, k, v)
    return o


def _lam_batch(lam):
    """Check a CUDA float64 Lambda batch [K, P], P = 13 or 16; returns it contiguous."""
    import torch
    if not (isinstance(lam, torch.Tensor) and lam.is_cuda and lam.dtype == torch.float64
            and lam.dim() == 2 and lam.shape[1] in (NUM_PARAMS, NUM_PARAMS_MULTIPEAK)):
        raise TypeError("lam must be a CUDA float64 tensor of shape [K, 13] (or [K, 16] for "
                        "the multi-peak model)")
    return lam.contiguous()


def _check_width(ctx, P):
    """The library reads P doubles per Lambda point from the context's mass model: refuse
    a batch of another width before it can read past the caller's tensor."""
    info = Info()
    _check(lib().gwc_get_info(ctx, ctypes.byref(info)), ctx)
    if P != info.n_params:
        raise TypeError(f"this context's mass model takes Lambda rows of {info.n_params} entries, not {P}")


def last_error(ctx=None) -> str:
    msg = lib().gwc_last_error(ctx)
    return msg.decode() if msg else ""


def _check(status, ctx=None):
    if status != 0:
        raise GwcError(status, last_error(ctx))


def _np_ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def create(cat: dict, options: Options | None = None, los_dtype_in: int = LOS_F32):
    """gwc_create from a catalogue dict of numpy arrays (see synth.catalogue)."""
    keep = {}

    def arr(key, dt):
        a = np.ascontiguousarray(cat[key], dtype=dt)
        keep[key] = a
        return _np_ptr(a)

    los = np.ascontiguousarray(cat["los"], dtype=np.uint16 if los_dtype_in == LOS_BF16 else np.float32)
    keep["los"] = los
    n_ev = len(cat["offsets"]) - 1
    ev = Events(n_events=n_ev, offsets=arr("offsets", np.int64), m1_det=arr("m1", np.float32),
                m2_det=arr("m2", np.float32), dl_mpc=arr("dl", np.float32),
                ln_pe_prior=arr("lnpe", np.float32), pix=arr("pix", np.int32))
    lo = Los(n_pix=los.shape[0], n_z=los.shape[1], z_max=float(cat["z_max"]), dtype=los_dtype_in,
             p_z=_np_ptr(los))
    inj = Injections(n_found=len(cat["inj_m1"]), n_draw=float(cat["n_draw"]),
                     m1_det=arr("inj_m1", np.float32), m2_det=arr("inj_m2", np.float32),
                     dl_mpc=arr("inj_dl", np.float32), ln_p_draw=arr("inj_lnpd", np.float32))
    out = ctypes.c_void_p()
    opt = options if options is not None else default_options()
    st = lib().gwc_create(ctypes.byref(ev), ctypes.byref(lo), ctypes.byref(inj), ctypes.byref(opt),
                          ctypes.byref(out))
    _check(st)
    return out


def destroy(ctx):
    lib().gwc_destroy(ctx)


def get_info(ctx) -> dict:
    info = Info()
    _check(lib().gwc_get_info(ctx, ctypes.byref(info)), ctx)
    return {f: getattr(info, f) for f, _ in Info._fields_}


def _outputs(K, n_ev, device, grad, P=NUM_PARAMS):
    import torch
    f64 = dict(dtype=torch.float64, device=device)
    out = dict(lnL_event=torch.empty((K, n_ev), **f64), neff_event=torch.empty((K, n_ev), **f64),
               ln_xi=torch.empty(K, **f64), neff_sel=torch.empty(K, **f64),
               lnL_total=torch.empty(K, **f64),
               flags=torch.empty(K, dtype=torch.int32, device=device))
    if grad:
        out["grad_total"] = torch.empty((K, P), **f64)
    return out


def _call(fn, ctx, lam, n_events, grad, stream, out, plain=False):
    lam = _lam_batch(lam)
    _check_width(ctx, lam.shape[1])
    K = lam.shape[0]
    if out is None:
        out = _outputs(K, n_events, lam.device, grad, lam.shape[1])
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    args = [ctx, K, p(lam), p(out["lnL_event"]), p(out["neff_event"]), p(out["ln_xi"]),
            p(out["neff_sel"]), p(out["lnL_total"]), p(out["flags"])]
    if grad or plain:
        args.append(p(out.get("grad_total")))
    args.append(_stream_ptr(stream))
    _check(fn(*args), ctx)
    return out


def loglik(ctx, lam, n_events, stream=None, out=None):
    """gwc_loglik: lam is a CUDA float64 tensor [K, P] (P = 13, or 16 for the multi-peak
    model, matching the context); returns a dict of tensors."""
    return _call(lib().gwc_loglik, ctx, lam, n_events, False, stream, out)


def loglik_grad(ctx, lam, n_events, stream=None, out=None):
    """gwc_loglik_grad: as loglik, plus grad_total [K, P]."""
    return _call(lib().gwc_loglik_grad, ctx, lam, n_events, True, stream, out)


def default_kde_options(**kw):
    o = KdeOptions()
    lib().gwc_default_kde_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "bw":
            k, v = "bw_rule", BW_RULES[v]
        setattr(o, k, v)
    return o


def loglik_kde(ctx, lam, n_events, bw="scott", n_grid=256, neff_min_pixel=2.0, stream=None, out=None):
    """gwc_loglik_kde: the paper's KDE form of the event terms (value only); neff_event
    holds the effective number of kept pixels of each event."""
    lam = _lam_batch(lam)
    _check_width(ctx, lam.shape[1])
    K = lam.shape[0]
    if out is None:
        out = _outputs(K, n_events, lam.device, False)
    o = default_kde_options(bw=bw, n_grid=n_grid, neff_min_pixel=neff_min_pixel)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(lib().gwc_loglik_kde(ctx, K, p(lam), ctypes.byref(o), p(out["lnL_event"]), p(out["neff_event"]),
                                p(out["ln_xi"]), p(out["neff_sel"]), p(out["lnL_total"]), p(out["flags"]),
                                _stream_ptr(stream)), ctx)
    return out


def loglik_plain(ctx, lam, n_events, grad=True, stream=None, out=None):
    """gwc_loglik_plain: the single-Lambda baseline path (same outputs)."""
    if out is None:
        import torch
        out = _outputs(lam.shape[0], n_events, lam.device, grad, lam.shape[-1])
        if not grad:
            out["grad_total"] = None
    return _call(lib().gwc_loglik_plain, ctx, lam, n_events, False, stream, out, plain=True)


def loglik_grad_host(ctx, lam: np.ndarray, grad=True, stream=None):
    """gwc_loglik_grad_host: host Lambda in, host total / flags / gradient out."""
    lam = np.ascontiguousarray(np.atleast_2d(lam), dtype=np.float64)
    _check_width(ctx, lam.shape[1])
    K = lam.shape[0]
    tot = np.empty(K, np.float64)
    flags = np.empty(K, np.int32)
    g = np.empty((K, lam.shape[1]), np.float64) if grad else None
    st = lib().gwc_loglik_grad_host(ctx, K, _np_ptr(lam), _np_ptr(tot), _np_ptr(flags),
                                    _np_ptr(g) if grad else None, _stream_ptr(stream))
    _check(st, ctx)
    return (tot, flags, g) if grad else (tot, flags)


def sample_terms(ctx, lam, n_total, grad=True, stream=None, cells=False):
    """gwc_sample_terms for one Lambda (CUDA float64 tensor [P]): (ln w - c, d [P, n], c[1 + P]),
    and with cells=True a fourth tensor, the int32 LOS grid cell of each sample (-1 where
    d_L maps outside [0, z_max])."""
    import torch
    lam = lam.contiguous()
    P = lam.numel()
    _check_width(ctx, P)
    lnw = torch.empty(n_total, dtype=torch.float32, device=lam.device)
    d = torch.empty((P, n_total), dtype=torch.float32, device=lam.device) if grad else None
    c = torch.empty(1 + P, dtype=torch.float64, device=lam.device)
    cell = torch.empty(n_total, dtype=torch.int32, device=lam.device) if cells else None
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    _check(lib().gwc_sample_terms(ctx, p(lam), p(lnw), p(d), p(c), p(cell), _stream_ptr(stream)), ctx)
    return (lnw, d, c, cell) if cells else (lnw, d, c)


def sample_terms_noalloc(lam, samples, pix, injections, los, z_max, n_x_table=512, grad=True,
                         stream=None):
    """gwc_sample_terms_noalloc on caller-owned CUDA tensors (no context, no allocation in
    the library): samples [n, 4] and injections [m, 4] float32, pix [n] int32, los
    [n_pix, n_z] float32, lam [13] float64, all contiguous and on the current CUDA device
    (the library reads them asynchronously on `stream`, so no temporary copy is made
    here).  Returns (ln w - c, d, c) like sample_terms; the output tensors are allocated
    here by PyTorch, not by the library."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())

    def need(t, name, dtype, dim, width=None):
        if not (isinstance(t, torch.Tensor) and t.device == dev and t.dtype == dtype and t.dim() == dim
                and (width is None or t.shape[-1] == width) and t.is_contiguous()):
            shape = f"[..., {width}]" if width else f"{dim}-D"
            raise TypeError(f"{name} must be a contiguous {dtype} {shape} tensor on {dev}")

    need(lam, "lam", torch.float64, 1, NUM_PARAMS)
    need(samples, "samples", torch.float32, 2, 4)
    need(pix, "pix", torch.int32, 1)
    need(injections, "injections", torch.float32, 2, 4)
    need(los, "los", torch.float32, 2)
    n, m = samples.shape[0], injections.shape[0]
    if pix.shape[0] != n:
        raise TypeError("pix must have one entry per sample")
    lnw = torch.empty(n + m, dtype=torch.float32, device=dev)
    d = torch.empty((NUM_PARAMS, n + m), dtype=torch.float32, device=dev) if grad else None
    c = torch.empty(1 + NUM_PARAMS, dtype=torch.float64, device=dev)
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    st = lib().gwc_sample_terms_noalloc(p(lam), n, p(samples), p(pix), m, p(injections),
                                        los.shape[0], los.shape[1], float(z_max), p(los), n_x_table,
                                        p(lnw), p(d), p(c), _stream_ptr(stream))
    _check(st)
    return lnw, d, c


CENSUS_SLOTS = ("live", "in_range", "mass_order", "support", "value", "value_win1", "value_win2",
                "weight", "weight_win1", "weight_win2")
UNITS = {"ffma": 0, "ffma2": 1, "ex2": 2, "lg2": 3, "rcp": 4, "rsqrt": 5, "dfma": 6, "dfma_lane1": 7}


def path_census(ctx, lam, stream=None):
    """gwc_path_census: how many (sample, Lambda) evaluations of the batch lam [K, P]
    reach each stage of the value arithmetic; returns a dict keyed by CENSUS_SLOTS."""
    import torch
    lam = _lam_batch(lam)
    _check_width(ctx, lam.shape[1])
    counts = torch.zeros(len(CENSUS_SLOTS), dtype=torch.int64, device=lam.device)
    _check(lib().gwc_path_census(ctx, lam.shape[0], ctypes.c_void_p(lam.data_ptr()),
                                 ctypes.c_void_p(counts.data_ptr()), _stream_ptr(stream)), ctx)
    return dict(zip(CENSUS_SLOTS, (int(v) for v in counts.cpu().numpy())))


KDE_CENSUS_SLOTS = ("pass1", "kept", "pass2", "terms")


def kde_census(ctx, lam, bw="scott", n_grid=256, neff_min_pixel=2.0, stream=None):
    """gwc_kde_census: the KDE kernel's work for the batch lam [K, P] (first-pass sample
    evaluations, kept groups, second-pass evaluations, grid terms); a dict keyed by
    KDE_CENSUS_SLOTS."""
    import torch
    lam = _lam_batch(lam)
    _check_width(ctx, lam.shape[1])
    counts = torch.zeros(len(KDE_CENSUS_SLOTS), dtype=torch.int64, device=lam.device)
    o = default_kde_options(bw=bw, n_grid=n_grid, neff_min_pixel=neff_min_pixel)
    _check(lib().gwc_kde_census(ctx, lam.shape[0], ctypes.c_void_p(lam.data_ptr()), ctypes.byref(o),
                                ctypes.c_void_p(counts.data_ptr()), _stream_ptr(stream)), ctx)
    return dict(zip(KDE_CENSUS_SLOTS, (int(v) for v in counts.cpu().numpy())))


def alu_probe(unit, blocks, iters, stream=None):
    """gwc_alu_probe: launch one throughput probe of an arithmetic unit (a key of UNITS)
    on the stream; returns the number of operations it performs (the caller times it)."""
    ops = ctypes.c_double(0.0)
    _check(lib().gwc_alu_probe(UNITS[unit], blocks, iters, ctypes.byref(ops), _stream_ptr(stream)))
    return ops.value


def _splitmix64_outputs(seed, k):
    """The (k+1)-th outputs of the SplitMix64 generator started at `seed` (uint64 arrays)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(k, dtype=np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def cap_selection(cat, cap, seed=0):
    """Input indices of the samples kept by the cap_per_pixel option (see include/gwc.h):
    in each (event, pixel) group larger than `cap`, the `cap` samples with the smallest
    SplitMix64 key; per event in input order.  Returns (indices, new offsets)."""
    off = np.asarray(cat["offsets"], dtype=np.int64)
    pix = np.asarray(cat["pix"])
    keep, counts = [], []
    for e in range(len(off) - 1):
        idx = np.arange(off[e], off[e + 1])
        sel = []
        for p in np.unique(pix[idx]):
            run = idx[pix[idx] == p]
            if cap > 0 and len(run) > cap:
                run = run[np.argsort(_splitmix64_outputs(seed, run), kind="stable")[:cap]]
            sel.append(run)
        sel = np.sort(np.concatenate(sel))
        keep.append(sel)
        counts.append(len(sel))
    return np.concatenate(keep), np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def capped(cat, cap, seed=0):
    """The catalogue as the library holds it under cap_per_pixel = cap, cap_seed = seed."""
    idx, off = cap_selection(cat, cap, seed)
    out = dict(cat)
    for k in ("m1", "m2", "dl", "lnpe", "pix"):
        out[k] = np.asarray(cat[k])[idx]
    out["offsets"] = off
    return out


def sample_order(cat):
    """Input index of each sample in the library's order (per event, stable sort by
    pixel id, then by d_L)."""
    off = np.asarray(cat["offsets"], dtype=np.int64)
    pix = np.asarray(cat["pix"])
    dl = np.asarray(cat["dl"], dtype=np.float32)
    out = []
    for e in range(len(off) - 1):
        idx = np.arange(off[e], off[e + 1])
        out.append(idx[np.lexsort((dl[idx], pix[idx]))])
    return np.concatenate(out) if out else np.zeros(0, np.int64)


INJ_BLOCK = 256


def injection_order(cat):
    """Input index of each injection in the library's order (stable sort by d_L, then
    each consecutive block of INJ_BLOCK stably sorted by detector-frame m1)."""
    order = np.argsort(np.asarray(cat["inj_dl"], dtype=np.float32), kind="stable")
    m1 = np.asarray(cat["inj_m1"], dtype=np.float32)[order]
    for a in range(0, len(order), INJ_BLOCK):
        order[a:a + INJ_BLOCK] = order[a:a + INJ_BLOCK][np.argsort(m1[a:a + INJ_BLOCK], kind="stable")]
    return order


def profile_enable(ctx, enable=True):
    """gwc_profile_enable: record per-stage CUDA events in every call."""
    _check(lib().gwc_profile_enable(ctx, int(bool(enable))), ctx)


def profile_read(ctx):
    """gwc_profile_read: (ms[prologue, samples, merge], n_calls) since the last read."""
    ms = np.zeros(3, np.float64)
    n = np.zeros(1, np.int64)
    _check(lib().gwc_profile_read(ctx, _np_ptr(ms), _np_ptr(n)), ctx)
    return ms, int(n[0])


def los_cell_index(z, n_z, z_max, stream=None):
    """gwc_los_cell_index on a CUDA float32 tensor; returns int32 cells (-1 outside)."""
    import torch
    z = z.contiguous()
    cell = torch.empty(z.shape, dtype=torch.int32, device=z.device)
    st = lib().gwc_los_cell_index(ctypes.c_void_p(z.data_ptr()), z.numel(), n_z, z_max,
                                  ctypes.c_void_p(cell.data_ptr()), _stream_ptr(stream))
    _check(st)
    return cell


class Graph:
    """gwc_graph: one recorded gwc_loglik / gwc_loglik_grad call on fixed tensors.

    ``lam`` [K, P] (CUDA float64) is the input the replays read: write the next points
    into it (``lam.copy_(...)``) and call ``launch()``; the results land in ``out``.
    """

    def __init__(self, context, lam, grad=True, out=None):
        import torch
        if not (isinstance(lam, torch.Tensor) and lam.is_contiguous()):
            raise TypeError("lam must be a contiguous CUDA float64 tensor of shape [K, P]")
        lam = _lam_batch(lam)
        _check_width(context._ctx, lam.shape[1])
        K = lam.shape[0]
        self.context, self.lam, self.grad = context, lam, grad
        self.out = out if out is not None else _outputs(K, context.n_events, lam.device, grad, lam.shape[1])
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        o = self.out
        h = ctypes.c_void_p()
        _check(lib().gwc_graph_create(context._ctx, K, p(lam), int(bool(grad)), p(o["lnL_event"]),
                                      p(o["neff_event"]), p(o["ln_xi"]), p(o["neff_sel"]),
                                      p(o["lnL_total"]), p(o["flags"]), p(o.get("grad_total")),
                                      ctypes.byref(h)), context._ctx)
        self._g = h

    def launch(self, stream=None):
        if self._g is None:
            raise GwcError(-1, "graph destroyed")
        _check(lib().gwc_graph_launch(self._g, _stream_ptr(stream)), None)
        return self.out

    def close(self):
        if self._g is not None:
            lib().gwc_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hmc:
    """gwc_hmc: one recorded HMC trajectory of n_leapfrog steps for K chains.

    The device tensors q, p, log_u (inputs) and lnL, grad, accept, H (outputs) are owned
    here; ``run(q, p, log_u)`` copies the inputs in (any of them may be omitted to keep
    the current contents) and replays the trajectory.  eps [K] and inv_mass [P] are
    fixed at creation (P: the context's Lambda width).
    """

    def __init__(self, context, K, n_leapfrog, eps, inv_mass, device="cuda"):
        import torch
        f64 = dict(dtype=torch.float64, device=device)
        self.context = context
        P = context.n_params
        self.eps = torch.as_tensor(eps, **f64).reshape(-1).expand(K).contiguous()
        self.inv_mass = torch.as_tensor(inv_mass, **f64).reshape(P).contiguous()
        self.q = torch.zeros((K, P), **f64)
        self.p = torch.zeros((K, P), **f64)
        self.log_u = torch.zeros(K, **f64)
        self.lnL = torch.zeros(K, **f64)
        self.grad = torch.zeros((K, P), **f64)
        self.accept = torch.zeros(K, dtype=torch.int32, device=device)
        self.H = torch.zeros((K, 2), **f64)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        h = ctypes.c_void_p()
        _check(lib().gwc_hmc_create(context._ctx, K, n_leapfrog, p(self.eps), p(self.inv_mass),
                                    p(self.q), p(self.p), p(self.log_u), p(self.lnL), p(self.grad),
                                    p(self.accept), p(self.H), ctypes.byref(h)), context._ctx)
        self._h = h

    def run(self, q=None, p=None, log_u=None, stream=None):
        if self._h is None:
            raise GwcError(-1, "hmc object destroyed")
        for dst, src in ((self.q, q), (self.p, p), (self.log_u, log_u)):
            if src is not None:
                dst.copy_(src)
        _check(lib().gwc_hmc_launch(self._h, _stream_ptr(stream)), None)
        return self

    def close(self):
        if self._h is not None:
            lib().gwc_hmc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A gwc_ctx: the catalogue resident on the device, evaluated at Lambda batches."""

    def __init__(self, cat: dict, options: Options | None = None, **opt_kw):
        if options is None:
            options = default_options(**opt_kw)
        self.options = options
        self.n_events = len(cat["offsets"]) - 1
        self._ctx = create(cat, options)
        self.n_params = NUM_PARAMS_MULTIPEAK if options.mass_model == MASS_MULTIPEAK else NUM_PARAMS

    def loglik(self, lam, stream=None):
        return loglik(self._ctx, lam, self.n_events, stream)

    def loglik_grad(self, lam, stream=None):
        return loglik_grad(self._ctx, lam, self.n_events, stream)

    def loglik_kde(self, lam, bw="scott", n_grid=256, neff_min_pixel=2.0, stream=None):
        return loglik_kde(self._ctx, lam, self.n_events, bw, n_grid, neff_min_pixel, stream)

    def loglik_parts(self, lam, grad=True, stream=None):
        """gwc_loglik_parts: this context's share of a sharded catalogue (see shard.merge_parts)."""
        import torch
        lam = _lam_batch(lam)
        _check_width(self._ctx, lam.shape[1])
        K, P = lam.shape
        f64 = dict(dtype=torch.float64, device=lam.device)
        out = _outputs(K, self.n_events, lam.device, False)
        del out["lnL_total"]
        out["sum_events"] = torch.empty(K, **f64)
        if grad:
            out["grad_events"] = torch.empty((K, P), **f64)
            out["grad_ln_xi"] = torch.empty((K, P), **f64)
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        _check(lib().gwc_loglik_parts(self._ctx, K, p(lam), p(out["lnL_event"]), p(out["neff_event"]),
                                      p(out["ln_xi"]), p(out["neff_sel"]), p(out["sum_events"]),
                                      p(out["flags"]), p(out.get("grad_events")), p(out.get("grad_ln_xi")),
                                      _stream_ptr(stream)), self._ctx)
        out["n_events"] = self.n_events
        return out

    def loglik_plain(self, lam, grad=True, stream=None):
        return loglik_plain(self._ctx, lam, self.n_events, grad, stream)

    def loglik_grad_host(self, lam, grad=True, stream=None):
        return loglik_grad_host(self._ctx, lam, grad, stream)

    def info(self):
        return get_info(self._ctx)

    def sample_terms(self, lam, grad=True, stream=None, cells=False):
        info = get_info(self._ctx)
        return sample_terms(self._ctx, lam, info["n_samples"] + info["n_injections"], grad, stream, cells)

    def path_census(self, lam, stream=None):
        return path_census(self._ctx, lam, stream)

    def kde_census(self, lam, bw="scott", n_grid=256, neff_min_pixel=2.0, stream=None):
        return kde_census(self._ctx, lam, bw, n_grid, neff_min_pixel, stream)

    def autotune(self, lam, grad=True, stream=None):
        """gwc_autotune on the Lambda batch lam [K, P]: returns the chosen shape."""
        lam = _lam_batch(lam)
        _check_width(self._ctx, lam.shape[1])
        r = TuneResult()
        _check(lib().gwc_autotune(self._ctx, lam.shape[0], ctypes.c_void_p(lam.data_ptr()),
                                  int(bool(grad)), _stream_ptr(stream), ctypes.byref(r)), self._ctx)
        return {"chunk": r.chunk, "lambda_tile": r.lambda_tile, "lambda_group": r.lambda_group,
                "n_tried": r.n_tried, "ms": r.ms}

    def hmc(self, K, n_leapfrog, eps, inv_mass):
        """Record an HMC trajectory of n_leapfrog steps for K chains (see Hmc)."""
        return Hmc(self, K, n_leapfrog, eps, inv_mass)

    def graph(self, lam, grad=True, out=None):
        """Record one call on these tensors as a CUDA graph (see Graph)."""
        return Graph(self, lam, grad, out)

    def profile_enable(self, enable=True):
        profile_enable(self._ctx, enable)

    def profile_read(self):
        return profile_read(self._ctx)

    def close(self):
        if self._ctx is not None:
            destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _autograd_function():
    import torch

    class GwcLogLik(torch.autograd.Function):
        """Total log-likelihood [K] of a Lambda batch; backward uses the fused gradient."""

        @staticmethod
        def forward(ctx, lam, context):
            out = context.loglik_grad(lam.detach())
            ctx.save_for_backward(out["grad_total"])
            return out["lnL_total"]

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out[:, None] * g, None

    return GwcLogLik


def __getattr__(name):
    if name == "GwcLogLik":
        fn = _autograd_function()
        globals()["GwcLogLik"] = fn
        return fn
    raise AttributeError(name)
