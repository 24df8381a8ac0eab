"""Python binding of libdotpe (dense GW likelihood on GB300, arXiv 2507.16022).

Argument marshalling only: every computation runs in the CUDA library behind
the C ABI declared in include/dotpe.h.  The functions keep the ABI's names.
Importing works without a GPU (the library only needs the CUDA runtime to
load); calls that need a device fail with DotpeError when there is none.
There is no CPU fallback: if libdotpe.so is missing the import raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdotpe.so")

# ---- constants mirrored from include/dotpe.h ---------------------------------
DOTPE_OK = 0
DOTPE_E_INVALID = -1
DOTPE_E_NOMEM = -2
DOTPE_E_ADMISSION = -3
DOTPE_E_NOT_READY = -4
DOTPE_E_TIMEOUT = -5
DOTPE_E_DEVICE = -6
DOTPE_E_NOT_FOUND = -7
DOTPE_E_UNSUPPORTED = -8

DOTPE_PREC_FP32, DOTPE_PREC_BF16, DOTPE_PREC_FP16, DOTPE_PREC_BF16X3 = 0, 1, 2, 3
DOTPE_PREC_FP16X3, DOTPE_PREC_MIXED = 4, 5
DOTPE_CONFIG_AUTOTUNE, DOTPE_CONFIG_NO_GRAPHS, DOTPE_CONFIG_NARROW_TILES = 0x1, 0x2, 0x4
DOTPE_CONFIG_SINGLE_CTA_TILES = 0x8
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "bf16x3": 3, "fp16x3": 4, "mixed": 5}
DOTPE_C128, DOTPE_C64 = 0, 1
DOTPE_FLAG_STORE_LNL = 0x1
DOTPE_FLAG_GEMM_ONLY = 0x2
DOTPE_FLAG_TEST_STALL = 0x100
DOTPE_STATE_QUEUED, DOTPE_STATE_RUNNING, DOTPE_STATE_DONE, DOTPE_STATE_FAILED = 0, 1, 2, 3
DOTPE_LNL_MARG, DOTPE_LNL_ML_MAX, DOTPE_ROW_MARGINAL, DOTPE_COL_MARGINAL = 0, 1, 2, 3

# Public C symbols (kept in sync with include/dotpe.h by a test).
SYMBOLS = ("dotpe_create", "dotpe_destroy", "dotpe_strerror", "dotpe_last_error_message",
           "dotpe_version", "dotpe_device_info", "dotpe_bank_load", "dotpe_bank_release",
           "dotpe_event_submit", "dotpe_event_poll", "dotpe_event_wait", "dotpe_evidence",
           "dotpe_lnl_blocks", "dotpe_event_release", "dotpe_dist_marg_eval",
           "dotpe_event_stream_wait", "dotpe_dist_marg_eval_noalloc", "dotpe_batch_submit",
           "dotpe_preselect", "dotpe_rb_weights", "dotpe_posterior_samples", "dotpe_bank_subset",
           "dotpe_bank_save", "dotpe_bank_open", "dotpe_evidence_merge")


class DotpeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


# ---- ctypes mirrors of the ABI structs ------------------------------------------
_dp = ctypes.POINTER(ctypes.c_double)


class dotpe_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64),
                ("n_slots", ctypes.c_int), ("flags", ctypes.c_int), ("max_batch", ctypes.c_int)]


class dotpe_bank_desc(ctypes.Structure):
    _fields_ = [("n_int", ctypes.c_int64), ("n_modes", ctypes.c_int),
                ("mode_m", ctypes.POINTER(ctypes.c_int)), ("n_bins", ctypes.c_int),
                ("f", _dp), ("w_quad", _dp), ("h", ctypes.c_void_p), ("h_dtype", ctypes.c_int),
                ("ln_w_int", _dp), ("pol", _dp), ("n_pol", ctypes.c_int)]


class dotpe_event_desc(ctypes.Structure):
    _fields_ = [("bank_id", ctypes.c_uint64), ("i0", ctypes.c_int64), ("i1", ctypes.c_int64),
                ("n_det", ctypes.c_int), ("psd", _dp), ("data", _dp), ("n_ext", ctypes.c_int64),
                ("t", _dp), ("R", _dp), ("ln_w_ext", _dp), ("n_phi", ctypes.c_int),
                ("u_min", ctypes.c_double), ("cut_delta", ctypes.c_double),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("block_rows", ctypes.c_int64), ("rb_dh", _dp), ("rb_hh", _dp), ("F", _dp)]


class dotpe_presel_desc(ctypes.Structure):
    _fields_ = [("bank_id", ctypes.c_uint64), ("i0", ctypes.c_int64), ("i1", ctypes.c_int64),
                ("n_det", ctypes.c_int), ("psd", _dp), ("data", _dp), ("n_t", ctypes.c_int),
                ("t_grid", _dp), ("n_phi", ctypes.c_int), ("delta", ctypes.c_double),
                ("precision", ctypes.c_int), ("flags", ctypes.c_int), ("rb_dh", _dp), ("rb_hh", _dp)]


class dotpe_rb_desc(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int), ("n_modes", ctypes.c_int), ("n_fine", ctypes.c_int64),
                ("f_fine", _dp), ("df_fine", _dp), ("psd", _dp), ("data", _dp), ("h0", _dp), ("t0", _dp),
                ("n_bins", ctypes.c_int), ("nodes", ctypes.POINTER(ctypes.c_int64))]


class dotpe_presel_out(ctypes.Structure):
    _fields_ = [("max_lnl_inco", ctypes.c_double), ("threshold", ctypes.c_double),
                ("arg_i", ctypes.c_int64), ("n_selected", ctypes.c_int64),
                ("kernel_ms", ctypes.c_float), ("device_ms", ctypes.c_float),
                ("device_status", ctypes.c_int32)]


class dotpe_event_stats(ctypes.Structure):
    _fields_ = [("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("footprint_bytes", ctypes.c_int64), ("device_ms", ctypes.c_float),
                ("prep_ms", ctypes.c_float), ("fused_ms", ctypes.c_float), ("refine_ms", ctypes.c_float),
                ("precision", ctypes.c_int), ("state", ctypes.c_int)]


class dotpe_evidence_out(ctypes.Structure):
    _fields_ = [("ln_z", ctypes.c_double), ("n_eff", ctypes.c_double),
                ("n_eff_int", ctypes.c_double), ("n_eff_ext", ctypes.c_double),
                ("max_lnl_ml", ctypes.c_double), ("arg_i", ctypes.c_int64),
                ("arg_e", ctypes.c_int64), ("arg_o", ctypes.c_int64),
                ("n_marginalised", ctypes.c_int64), ("n_pairs", ctypes.c_int64),
                ("lnl_ml_threshold", ctypes.c_double), ("device_status", ctypes.c_int32),
                ("n_refined_tiles", ctypes.c_int32),
                ("n_screen_candidates", ctypes.c_int64), ("n_screen_evaluated", ctypes.c_int64)]


class dotpe_shard(ctypes.Structure):
    _fields_ = [("ev", dotpe_evidence_out), ("n_int", ctypes.c_int64), ("ln_p_ext", ctypes.POINTER(ctypes.c_double))]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libdotpe.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with paper_2507_16022_gb300._build.build()")
    L = ctypes.CDLL(path)
    vp, u64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "dotpe_create": ([ctypes.POINTER(dotpe_config), ctypes.POINTER(vp)], ctypes.c_int),
        "dotpe_destroy": ([vp], ctypes.c_int),
        "dotpe_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "dotpe_last_error_message": ([], ctypes.c_char_p),
        "dotpe_version": ([], ctypes.c_int),
        "dotpe_device_info": ([vp, ctypes.POINTER(ctypes.c_int), ctypes.c_char_p, ctypes.c_int],
                              ctypes.c_int),
        "dotpe_bank_load": ([vp, ctypes.POINTER(dotpe_bank_desc), u64p], ctypes.c_int),
        "dotpe_bank_release": ([vp, ctypes.c_uint64], ctypes.c_int),
        "dotpe_bank_subset": ([vp, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int64, u64p], ctypes.c_int),
        "dotpe_bank_save": ([vp, ctypes.c_uint64, ctypes.c_char_p], ctypes.c_int),
        "dotpe_bank_open": ([vp, ctypes.c_char_p, u64p], ctypes.c_int),
        "dotpe_event_submit": ([vp, ctypes.POINTER(dotpe_event_desc), u64p], ctypes.c_int),
        "dotpe_batch_submit": ([vp, ctypes.c_int, ctypes.POINTER(dotpe_event_desc), u64p], ctypes.c_int),
        "dotpe_event_poll": ([vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(dotpe_event_stats)], ctypes.c_int),
        "dotpe_event_wait": ([vp, ctypes.c_uint64, ctypes.c_double], ctypes.c_int),
        "dotpe_evidence": ([vp, ctypes.c_uint64, ctypes.POINTER(dotpe_evidence_out)], ctypes.c_int),
        "dotpe_lnl_blocks": ([vp, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                              ctypes.c_int64, ctypes.c_int, vp, ctypes.c_int64], ctypes.c_int),
        "dotpe_event_release": ([vp, ctypes.c_uint64], ctypes.c_int),
        "dotpe_dist_marg_eval": ([vp, ctypes.c_int64, vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "dotpe_event_stream_wait": ([vp, ctypes.c_uint64, vp], ctypes.c_int),
        "dotpe_dist_marg_eval_noalloc": ([vp, ctypes.c_int64, vp, vp, ctypes.c_float, vp], ctypes.c_int),
        "dotpe_preselect": ([vp, ctypes.POINTER(dotpe_presel_desc), vp, vp, vp, vp,
                             ctypes.POINTER(dotpe_presel_out)], ctypes.c_int),
        "dotpe_rb_weights": ([vp, ctypes.POINTER(dotpe_rb_desc), vp, vp], ctypes.c_int),
        "dotpe_posterior_samples": ([vp, ctypes.c_uint64, ctypes.c_int64, vp, vp, vp, vp, vp], ctypes.c_int),
        "dotpe_evidence_merge": ([ctypes.c_int, ctypes.POINTER(dotpe_shard), ctypes.c_int64, ctypes.c_int,
                                  ctypes.POINTER(dotpe_evidence_out), vp], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(status):
    if status != DOTPE_OK:
        L = load()
        raise DotpeError(status, f"{L.dotpe_strerror(status).decode()}: "
                                 f"{L.dotpe_last_error_message().decode()}")
    return status


def _ptr(a, ctype=ctypes.c_double):
    """Pointer to a contiguous numpy array (host) or an int device address."""
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.cast(ctypes.c_void_p(a), ctypes.POINTER(ctype))
    if hasattr(a, "data_ptr"):  # torch tensor
        return ctypes.cast(ctypes.c_void_p(a.data_ptr()), ctypes.POINTER(ctype))
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _host_c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


# ---- thin wrappers with the ABI's names ---------------------------------------
def dotpe_create(device=0, hbm_budget_bytes=0, n_slots=0, flags=0, max_batch=0):
    L = load()
    cfg = dotpe_config(device, hbm_budget_bytes, n_slots, flags, max_batch)
    h = ctypes.c_void_p()
    _check(L.dotpe_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def dotpe_destroy(ctx):
    return _check(load().dotpe_destroy(ctx))


def dotpe_version():
    return load().dotpe_version()


def dotpe_device_info(ctx):
    n = ctypes.c_int()
    buf = ctypes.create_string_buffer(256)
    _check(load().dotpe_device_info(ctx, ctypes.byref(n), buf, 256))
    return n.value, buf.value.decode()


def dotpe_bank_load(ctx, h, f, w_quad, mode_m, ln_w_int=None, pol=None):
    """h: [I, M, B] complex128/complex64 numpy array, or a torch tensor on the device
    (complex128/complex64, contiguous); [I, M, 2, B] is a polarisation-resolved
    (precessing) bank h_{impb}, whose events take antenna patterns F.  pol:
    optional [I, M, 2] complex polarisation factors K_{imp} (needed by
    dotpe_preselect)."""
    L = load()
    keep = []
    if hasattr(h, "data_ptr"):
        import torch
        dtype = DOTPE_C128 if h.dtype == torch.complex128 else DOTPE_C64
        I, M, B = h.shape[0], h.shape[1], h.shape[-1]
        hp = ctypes.c_void_p(h.data_ptr())
    else:
        if h.dtype == np.complex64:
            h = np.ascontiguousarray(h)
            dtype = DOTPE_C64
        else:
            h = _host_c128(h)
            dtype = DOTPE_C128
        I, M, B = h.shape[0], h.shape[1], h.shape[-1]
        hp = ctypes.c_void_p(h.ctypes.data)
        keep.append(h)
    if len(h.shape) == 4 and h.shape[2] != 2:
        raise ValueError(f"a polarisation-resolved bank is [I, M, 2, B], got {tuple(h.shape)}")
    n_pol = 2 if len(h.shape) == 4 else 1
    mm = np.ascontiguousarray(mode_m, dtype=np.int32)
    f = np.ascontiguousarray(f, dtype=np.float64)
    w = np.ascontiguousarray(w_quad, dtype=np.float64)
    lw = None if ln_w_int is None else np.ascontiguousarray(ln_w_int, dtype=np.float64)
    pl = None if pol is None else _host_c128(pol)
    if pl is not None and pl.shape != (I, M, 2):
        raise ValueError(f"pol has shape {pl.shape}, expected {(I, M, 2)}")
    desc = dotpe_bank_desc(I, M, mm.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), B, _ptr(f), _ptr(w),
                           hp, dtype, _ptr(lw), None if pl is None else _ptr(pl.view(np.float64)), n_pol)
    bid = ctypes.c_uint64()
    _check(L.dotpe_bank_load(ctx, ctypes.byref(desc), ctypes.byref(bid)))
    return bid.value


def dotpe_bank_subset(ctx, bank_id, rows):
    """A new bank of the rows (int64, numpy host array or torch tensor on the device)
    of bank_id, e.g. the pre-selection's `selected` rows."""
    if hasattr(rows, "data_ptr"):
        ptr, n = ctypes.c_void_p(rows.data_ptr()), int(rows.numel())
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        ptr, n = ctypes.c_void_p(rows.ctypes.data), int(rows.shape[0])
    bid = ctypes.c_uint64()
    _check(load().dotpe_bank_subset(ctx, ctypes.c_uint64(bank_id), ptr, n, ctypes.byref(bid)))
    return bid.value


def dotpe_bank_save(ctx, bank_id, path):
    """Write the bank to a file (checkpoint)."""
    return _check(load().dotpe_bank_save(ctx, ctypes.c_uint64(bank_id), os.fsencode(path)))


def dotpe_bank_open(ctx, path):
    """Load a bank file written by dotpe_bank_save as a new bank; returns its id."""
    bid = ctypes.c_uint64()
    _check(load().dotpe_bank_open(ctx, os.fsencode(path), ctypes.byref(bid)))
    return bid.value


def dotpe_bank_release(ctx, bank_id):
    return _check(load().dotpe_bank_release(ctx, bank_id))


def _event_desc(keep, bank_id, i0, i1, psd, data, t, R, ln_w_ext=None, n_phi=32, u_min=1.0,
                cut_delta=0.0, precision="bf16x3", flags=0, stream=None, block_rows=0, rb=None, F=None):

    def arr(a, cplx=False):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            keep.append(a)
            return _ptr(a)
        a = _host_c128(a) if cplx else np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        return _ptr(a.view(np.float64) if cplx else a)

    D = t.shape[1]
    E = t.shape[0]
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    rbd, rbh = (None, None) if rb is None else (arr(rb[0], True), arr(rb[1], True))
    return dotpe_event_desc(bank_id, i0, i1, D, arr(psd), arr(data, True), E, arr(t), arr(R, True),
                            arr(ln_w_ext), n_phi, u_min, cut_delta, prec, flags, st, block_rows, rbd, rbh,
                            arr(F))


def dotpe_event_submit(ctx, bank_id, i0, i1, psd, data, t, R, ln_w_ext=None, n_phi=32, u_min=1.0,
                       cut_delta=0.0, precision="bf16x3", flags=0, stream=None, block_rows=0, rb=None, F=None):
    """psd [D,B], data [D,B] complex, t [E,D], R [E,D,M] complex, ln_w_ext [E]: numpy (host)
    or torch tensors (host or device; complex tensors as float64 views are accepted).
    block_rows: 0, or a multiple of 128 to stream the slice through in bank blocks.
    rb: optional (w_dh [D,M,B], w_hh [D,M,M,B]) relative-binning weights (psd, data may be None).
    F: [E,D,2] real antenna patterns, for a polarisation-resolved bank (R may then be None)."""
    keep = []
    desc = _event_desc(keep, bank_id, i0, i1, psd, data, t, R, ln_w_ext, n_phi, u_min, cut_delta,
                       precision, flags, stream, block_rows, rb, F)
    eid = ctypes.c_uint64()
    _check(load().dotpe_event_submit(ctx, ctypes.byref(desc), ctypes.byref(eid)))
    return eid.value


def dotpe_batch_submit(ctx, specs):
    """specs: list of dicts of dotpe_event_submit's keyword arguments (bank_id, i0, i1, psd,
    data, t, R, ...), one per event; all share the bank and the precision.  Returns the ids."""
    keep = []
    n = len(specs)
    descs = (dotpe_event_desc * n)(*[_event_desc(keep, **sp) for sp in specs])
    ids = (ctypes.c_uint64 * n)()
    _check(load().dotpe_batch_submit(ctx, n, descs, ids))
    return list(ids)


def dotpe_event_poll(ctx, event_id):
    st = ctypes.c_int()
    s = dotpe_event_stats()
    _check(load().dotpe_event_poll(ctx, event_id, ctypes.byref(st), ctypes.byref(s)))
    return st.value, {k: getattr(s, k) for k, _ in s._fields_}


def dotpe_event_wait(ctx, event_id, timeout_s=0.0):
    return _check(load().dotpe_event_wait(ctx, event_id, timeout_s))


def dotpe_event_stream_wait(ctx, event_id, stream):
    """stream: torch.cuda.Stream or a raw cudaStream_t integer."""
    st = stream if isinstance(stream, int) else stream.cuda_stream
    return _check(load().dotpe_event_stream_wait(ctx, event_id, ctypes.c_void_p(st)))


def dotpe_evidence(ctx, event_id):
    o = dotpe_evidence_out()
    _check(load().dotpe_evidence(ctx, event_id, ctypes.byref(o)))
    return {k: getattr(o, k) for k, _ in o._fields_}


def dotpe_evidence_merge(shards, n_phi):
    """shards: list of (evidence dict as dotpe_evidence returns it, n_int, ln_p_ext [n_ext]),
    one per bank-row shard of one event.  Returns (evidence dict, ln_p_ext [n_ext] float64)."""
    n = len(shards)
    keep = [np.ascontiguousarray(lp, dtype=np.float64) for _, _, lp in shards]
    n_ext = keep[0].shape[0] if n else 0
    arr = (dotpe_shard * max(n, 1))()
    for k, (ev, n_int, _) in enumerate(shards):
        e = dotpe_evidence_out()
        for name, _ in e._fields_:
            # the screening counters are diagnostics: -1 (not counted) when absent
            setattr(e, name, ev.get(name, -1) if name.startswith("n_screen") else ev[name])
        arr[k].ev = e
        arr[k].n_int = int(n_int)
        arr[k].ln_p_ext = keep[k].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    o = dotpe_evidence_out()
    out = np.zeros(max(n_ext, 1))
    _check(load().dotpe_evidence_merge(n, arr, n_ext, int(n_phi), ctypes.byref(o), _ptr(out)))
    return {k: getattr(o, k) for k, _ in o._fields_}, out[:n_ext]


def dotpe_lnl_blocks(ctx, event_id, i0, i1, e0, e1, what=DOTPE_LNL_MARG, out=None):
    """Returns a float32 array (host) unless `out` (numpy or torch) is given."""
    L = load()
    if what in (DOTPE_ROW_MARGINAL, DOTPE_COL_MARGINAL):
        n = (i1 - i0) if what == DOTPE_ROW_MARGINAL else (e1 - e0)
        shape, ld = (n,), n
    else:
        shape, ld = (i1 - i0, e1 - e0), e1 - e0
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    p = ctypes.c_void_p(out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data)
    _check(L.dotpe_lnl_blocks(ctx, event_id, i0, i1, e0, e1, what, p, ld))
    return out


def dotpe_event_release(ctx, event_id):
    return _check(load().dotpe_event_release(ctx, event_id))


def dotpe_posterior_samples(ctx, event_id, uniforms):
    """Posterior samples of a finished event (stored with DOTPE_FLAG_STORE_LNL);
    uniforms [n, 4] in [0, 1).  Returns (i, e, o, d_L / d_L^0) numpy arrays."""
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    n = u.shape[0]
    i = np.empty(n, np.int64)
    e = np.empty(n, np.int64)
    o = np.empty(n, np.int32)
    d = np.empty(n, np.float64)
    _check(load().dotpe_posterior_samples(ctx, event_id, n, ctypes.c_void_p(u.ctypes.data),
                                          ctypes.c_void_p(i.ctypes.data), ctypes.c_void_p(e.ctypes.data),
                                          ctypes.c_void_p(o.ctypes.data), ctypes.c_void_p(d.ctypes.data)))
    return i, e, o, d


def dotpe_rb_weights(ctx, f_fine, df_fine, psd, data, h0, nodes, t0=None):
    """Relative-binning weights (App. A) on the device: f_fine, df_fine [N], psd [D,N],
    data [D,N] complex, h0 [M,N] complex, nodes [B] int64, t0 [D] (numpy, host).
    Returns (w_dh [D,M,B], w_hh [D,M,M,B]) complex128."""
    f_fine = np.ascontiguousarray(f_fine, dtype=np.float64)
    df_fine = np.ascontiguousarray(df_fine, dtype=np.float64)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    data = _host_c128(data)
    h0 = _host_c128(h0)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    t0 = None if t0 is None else np.ascontiguousarray(t0, dtype=np.float64)
    D, N = psd.shape
    M, B = h0.shape[0], nodes.shape[0]
    w_dh = np.zeros((D, M, B), np.complex128)
    w_hh = np.zeros((D, M, M, B), np.complex128)
    desc = dotpe_rb_desc(D, M, N, _ptr(f_fine), _ptr(df_fine), _ptr(psd), _ptr(data.view(np.float64)),
                         _ptr(h0.view(np.float64)), _ptr(t0), B, nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    _check(load().dotpe_rb_weights(ctx, ctypes.byref(desc), ctypes.c_void_p(w_dh.ctypes.data),
                                   ctypes.c_void_p(w_hh.ctypes.data)))
    return w_dh, w_hh


def dotpe_preselect(ctx, bank_id, i0, i1, psd, data, t_grid, n_phi=32, delta=20.0, precision="fp16x3",
                    outputs=("lnl_ml", "arg_ot", "lnl_inco", "selected"), rb=None):
    """Incoherent single-detector pre-selection (Sec. IV.D, App. B) of bank rows [i0, i1).

    psd [D, B], data [D, B] complex, t_grid [D, n_t] (numpy, host).  Returns a dict
    with the dotpe_presel_out fields and the requested host arrays: lnl_ml [N, D]
    float32, arg_ot [N, D, 2] int32 ((o, t)), lnl_inco [N] float64, selected
    [n_selected] int64 (slice-relative rows)."""
    L = load()
    psd = None if psd is None else np.ascontiguousarray(psd, dtype=np.float64)
    data = None if data is None else _host_c128(data)
    tg = np.ascontiguousarray(t_grid, dtype=np.float64)
    D, n_t = tg.shape
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    rbd = rbh = None
    if rb is not None:
        rbd, rbh = _host_c128(rb[0]), _host_c128(rb[1])
    desc = dotpe_presel_desc(bank_id, i0, i1, D, _ptr(psd), None if data is None else _ptr(data.view(np.float64)),
                             n_t, _ptr(tg), n_phi, float(delta), prec, 0,
                             None if rbd is None else _ptr(rbd.view(np.float64)),
                             None if rbh is None else _ptr(rbh.view(np.float64)))
    N = i1 - i0
    arrs = {}
    if "lnl_ml" in outputs:
        arrs["lnl_ml"] = np.empty((N, D), dtype=np.float32)
    if "arg_ot" in outputs:
        arrs["arg_ot"] = np.empty((N, D, 2), dtype=np.int32)
    if "lnl_inco" in outputs:
        arrs["lnl_inco"] = np.empty(N, dtype=np.float64)
    if "selected" in outputs:
        arrs["selected"] = np.empty(N, dtype=np.int64)
    vp = lambda k: ctypes.c_void_p(arrs[k].ctypes.data) if k in arrs else None
    o = dotpe_presel_out()
    _check(L.dotpe_preselect(ctx, ctypes.byref(desc), vp("lnl_ml"), vp("arg_ot"), vp("lnl_inco"),
                             vp("selected"), ctypes.byref(o)))
    res = {k: getattr(o, k) for k, _ in o._fields_}
    if "selected" in arrs:
        arrs["selected"] = arrs["selected"][:o.n_selected]
    res.update(arrs)
    return res


def dotpe_dist_marg_eval(ctx, dh, hh, u_min):
    dh = np.ascontiguousarray(dh, dtype=np.float32)
    hh = np.ascontiguousarray(hh, dtype=np.float32)
    out = np.empty_like(dh)
    _check(load().dotpe_dist_marg_eval(ctx, dh.size, ctypes.c_void_p(dh.ctypes.data),
                                       ctypes.c_void_p(hh.ctypes.data), float(u_min),
                                       ctypes.c_void_p(out.ctypes.data)))
    return out


DIST_MARG_NOALLOC_MAX = 1 << 20


def dotpe_dist_marg_eval_noalloc(ctx, dh, hh, u_min):
    """Same values as dotpe_dist_marg_eval, through the allocation-free entry point
    (its scratch is a static device array; at most 2^20 values per call)."""
    dh = np.ascontiguousarray(dh, dtype=np.float32)
    hh = np.ascontiguousarray(hh, dtype=np.float32)
    out = np.empty_like(dh)
    _check(load().dotpe_dist_marg_eval_noalloc(ctx, dh.size, ctypes.c_void_p(dh.ctypes.data),
                                               ctypes.c_void_p(hh.ctypes.data), float(u_min),
                                               ctypes.c_void_p(out.ctypes.data)))
    return out
