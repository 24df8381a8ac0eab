"""FP64 CPU oracle (ctypes wrapper around oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may use it; the library path never does.  It
shares no code with the CUDA library.  Every function cites the passage of
arXiv 2507.16022 it follows (see oracle.h).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (portable flags: x86_64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [("n_int", ctypes.c_int), ("n_ext", ctypes.c_int), ("n_det", ctypes.c_int),
                ("n_modes", ctypes.c_int), ("n_bins", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("mode_m", ctypes.POINTER(ctypes.c_int)),
                ("f", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
                ("psd", ctypes.POINTER(ctypes.c_double)), ("data", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)), ("R", ctypes.POINTER(ctypes.c_double)),
                ("t", ctypes.POINTER(ctypes.c_double)),
                ("ln_w_int", ctypes.POINTER(ctypes.c_double)),
                ("ln_w_ext", ctypes.POINTER(ctypes.c_double)),
                ("u_min", ctypes.c_double),
                ("rb_dh", ctypes.POINTER(ctypes.c_double)), ("rb_hh", ctypes.POINTER(ctypes.c_double)),
                ("n_pol", ctypes.c_int), ("F", ctypes.POINTER(ctypes.c_double))]


PAIR_DTYPE = np.dtype([("lnl_marg", "f8"), ("lnl_sq", "f8"), ("lnl_ml_max", "f8"),
                       ("argmax_o", "i4"), ("n_pass", "i4")])


class EvidenceOut(ctypes.Structure):
    _fields_ = [("ln_z", ctypes.c_double), ("n_eff", ctypes.c_double),
                ("n_eff_int", ctypes.c_double), ("n_eff_ext", ctypes.c_double),
                ("max_lnl_ml", ctypes.c_double), ("arg_i", ctypes.c_int64),
                ("arg_e", ctypes.c_int64), ("arg_o", ctypes.c_int64),
                ("n_marginalised", ctypes.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_dist_marg.restype = ctypes.c_double
            L.or_dist_marg.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.or_lnl_ml.restype = ctypes.c_double
            L.or_lnl_ml.argtypes = [ctypes.c_double, ctypes.c_double]
            L.or_default_threads.restype = ctypes.c_int
            L.or_dist_sample.restype = ctypes.c_double
            L.or_dist_sample.argtypes = [ctypes.c_double] * 4
            L.or_quad_ml.restype = ctypes.c_double
            L.or_quad_ml.argtypes = [ctypes.c_double] * 5
            for name in ("or_data_weights", "or_direct_phases", "or_mode_components",
                         "or_rotate_phases", "or_eval_pairs", "or_eval_grid",
                         "or_direct_grid_ml", "or_evidence", "or_presel_grid", "or_presel",
                         "or_rb_weights"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a


class OracleProblem:
    """Holds contiguous FP64 copies of one workload and the ctypes struct."""

    def __init__(self, bank, ext, event, i_slice=None, rb=None):
        """rb: optional (w_dh [D, J, B], w_hh [D, J, J, B]) relative-binning weights (App. A,
        Eqs. dh_weights, hh_weights), one per (mode, polarisation) component: J = M for a
        mode bank, J = 2M (index 2m + p) for a polarisation-resolved bank."""
        h = bank.h if i_slice is None else bank.h[i_slice]
        lw_i = bank.ln_w if i_slice is None else bank.ln_w[i_slice]
        self.mode_m = np.ascontiguousarray(bank.mode_m, dtype=np.int32)
        self.f = np.ascontiguousarray(bank.f, dtype=np.float64)
        self.w = np.ascontiguousarray(bank.w, dtype=np.float64)
        self.psd = np.ascontiguousarray(event.psd, dtype=np.float64)
        self.data = _c128(event.data)
        self.h = _c128(h)
        # polarisation-resolved bank: h [I, M, 2, B] with real antenna patterns ext.F [E, D, 2]
        self.n_pol = 2 if self.h.ndim == 4 else 1
        self.R = _c128(ext.R) if self.n_pol == 1 else np.zeros(1, np.complex128)
        self.F = (np.ascontiguousarray(ext.F, dtype=np.float64) if self.n_pol == 2 else None)
        self.t = np.ascontiguousarray(ext.t, dtype=np.float64)
        self.ln_w_int = np.ascontiguousarray(lw_i, dtype=np.float64)
        self.ln_w_ext = np.ascontiguousarray(ext.ln_w, dtype=np.float64)
        I, M, B = self.h.shape[0], self.h.shape[1], self.h.shape[-1]
        E, D = self.t.shape
        self.shape = (I, E, D, M, B)
        self.n_phi = int(event.n_phi)
        self.u_min = float(event.u_min)
        self.rb = None if rb is None else (_c128(rb[0]), _c128(rb[1]))
        if self.rb is not None:
            J = M * self.n_pol
            assert self.rb[0].shape == (D, J, B) and self.rb[1].shape == (D, J, J, B)
        self.s = Problem(I, E, D, M, B, self.n_phi,
                         self.mode_m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         _dp(self.f), _dp(self.w), _dp(self.psd), _dp(self.data.view(np.float64)),
                         _dp(self.h.view(np.float64)), _dp(self.R.view(np.float64)), _dp(self.t),
                         _dp(self.ln_w_int), _dp(self.ln_w_ext), self.u_min,
                         None if rb is None else _dp(self.rb[0].view(np.float64)),
                         None if rb is None else _dp(self.rb[1].view(np.float64)),
                         self.n_pol, None if self.F is None else _dp(self.F))

    # -- components -------------------------------------------------------
    def data_weights(self):
        """Eq. inner_product: c_{d,b} = 4 w conj(d)/S, omega = 4 w / S."""
        I, E, D, M, B = self.shape
        c = np.zeros((D, B), np.complex128)
        om = np.zeros((D, B))
        lib().or_data_weights(D, B, _dp(self.w), _dp(self.psd), _dp(self.data.view(np.float64)),
                              _dp(c.view(np.float64)), _dp(om))
        return c, om

    def direct_phases(self, i, e):
        """Route O1: (dh_o, hh_o) for o = 0..n_phi-1 by the direct frequency sum."""
        dh = np.zeros(self.n_phi)
        hh = np.zeros(self.n_phi)
        lib().or_direct_phases(ctypes.byref(self.s), ctypes.c_int64(i), ctypes.c_int64(e),
                               _dp(dh), _dp(hh))
        return dh, hh

    def mode_components(self, i, e):
        """Route O2: z_m [M] and H_{mm'} [M, M] (complex)."""
        I, E, D, M, B = self.shape
        c, om = self.data_weights()
        z = np.zeros(M, np.complex128)
        H = np.zeros((M, M), np.complex128)
        lib().or_mode_components(ctypes.byref(self.s), _dp(c.view(np.float64)), _dp(om),
                                 ctypes.c_int64(i), ctypes.c_int64(e), _dp(z.view(np.float64)),
                                 _dp(H.view(np.float64)))
        return z, H

    def rotate_phases(self, z, H, n_phi=None):
        n_phi = self.n_phi if n_phi is None else n_phi
        M = self.shape[3]
        z = _c128(z)
        H = _c128(H)
        dh = np.zeros(n_phi)
        hh = np.zeros(n_phi)
        lib().or_rotate_phases(M, self.mode_m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               _dp(z.view(np.float64)), _dp(H.view(np.float64)), n_phi,
                               _dp(dh), _dp(hh))
        return dh, hh

    # -- evaluation -------------------------------------------------------
    def eval_pairs(self, pi, pe, threshold=-np.inf, n_threads=0):
        pi = np.ascontiguousarray(pi, dtype=np.int64)
        pe = np.ascontiguousarray(pe, dtype=np.int64)
        out = np.zeros(pi.shape[0], dtype=PAIR_DTYPE)
        lib().or_eval_pairs(ctypes.byref(self.s), ctypes.c_int64(pi.shape[0]),
                            pi.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            pe.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                            ctypes.c_double(threshold), n_threads,
                            out.ctypes.data_as(ctypes.c_void_p))
        return out

    def eval_grid(self, cut_delta=0.0, n_threads=0):
        I, E = self.shape[:2]
        out = np.zeros(I * E, dtype=PAIR_DTYPE)
        thr = ctypes.c_double(0.0)
        lib().or_eval_grid(ctypes.byref(self.s), ctypes.c_double(cut_delta), n_threads,
                           out.ctypes.data_as(ctypes.c_void_p), ctypes.byref(thr))
        return out.reshape(I, E), thr.value

    def direct_grid_ml(self, n_threads=0):
        I, E = self.shape[:2]
        out = np.zeros(I * E)
        lib().or_direct_grid_ml(ctypes.byref(self.s), n_threads, _dp(out))
        return out.reshape(I, E)

    def evidence(self, grid):
        I, E = self.shape[:2]
        g = np.ascontiguousarray(grid.reshape(-1), dtype=PAIR_DTYPE)
        ev = EvidenceOut()
        lpi = np.zeros(I)
        lpe = np.zeros(E)
        lib().or_evidence(ctypes.byref(self.s), g.ctypes.data_as(ctypes.c_void_p),
                          ctypes.byref(ev), _dp(lpi), _dp(lpe))
        return dict(ln_z=ev.ln_z, n_eff=ev.n_eff, n_eff_int=ev.n_eff_int,
                    n_eff_ext=ev.n_eff_ext, max_lnl_ml=ev.max_lnl_ml,
                    arg=(ev.arg_i, ev.arg_e, ev.arg_o), n_marginalised=ev.n_marginalised,
                    ln_p_int=lpi, ln_p_ext=lpe)


class PreselStruct(ctypes.Structure):
    _fields_ = [("n_int", ctypes.c_int), ("n_det", ctypes.c_int), ("n_modes", ctypes.c_int),
                ("n_bins", ctypes.c_int), ("n_t", ctypes.c_int), ("n_phi", ctypes.c_int),
                ("mode_m", ctypes.POINTER(ctypes.c_int)),
                ("f", ctypes.POINTER(ctypes.c_double)), ("w", ctypes.POINTER(ctypes.c_double)),
                ("psd", ctypes.POINTER(ctypes.c_double)), ("data", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)), ("pol", ctypes.POINTER(ctypes.c_double)),
                ("t_grid", ctypes.POINTER(ctypes.c_double)),
                ("rb_dh", ctypes.POINTER(ctypes.c_double)), ("rb_hh", ctypes.POINTER(ctypes.c_double)),
                ("n_pol", ctypes.c_int)]


class PreselProblem:
    """Incoherent single-detector pre-selection (Sec. IV.D, App. B) of one event
    over bank rows: h [I, M, B] with pol [I, M, 2] (K_{imp}, p = +, x), or a
    polarisation-resolved bank h [I, M, 2, B] (pol None); t_grid [D, n_t]."""

    def __init__(self, f, w, mode_m, h, pol, psd, data, t_grid, n_phi=32, rb=None):
        self.mode_m = np.ascontiguousarray(mode_m, dtype=np.int32)
        self.f = np.ascontiguousarray(f, dtype=np.float64)
        self.w = np.ascontiguousarray(w, dtype=np.float64)
        self.h = _c128(h)
        self.n_pol = 2 if self.h.ndim == 4 else 1
        self.pol = _c128(pol) if self.n_pol == 1 else np.zeros(1, np.complex128)
        self.psd = np.ascontiguousarray(psd, dtype=np.float64)
        self.data = _c128(data)
        self.t_grid = np.ascontiguousarray(t_grid, dtype=np.float64)
        I, M, B = self.h.shape[0], self.h.shape[1], self.h.shape[-1]
        D, NT = self.t_grid.shape
        assert self.n_pol == 1 or self.h.shape[2] == 2
        assert (self.n_pol == 2 or self.pol.shape == (I, M, 2)) and self.psd.shape == (D, B) \
            and self.data.shape == (D, B)
        self.shape = (I, D, M, B, NT)
        self.n_phi = int(n_phi)
        self.rb = None if rb is None else (_c128(rb[0]), _c128(rb[1]))
        J = M * self.n_pol
        assert rb is None or (self.rb[0].shape == (D, J, B) and self.rb[1].shape == (D, J, J, B))
        self.s = PreselStruct(I, D, M, B, NT, self.n_phi,
                              self.mode_m.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                              _dp(self.f), _dp(self.w), _dp(self.psd), _dp(self.data.view(np.float64)),
                              _dp(self.h.view(np.float64)), _dp(self.pol.view(np.float64)),
                              _dp(self.t_grid),
                              None if rb is None else _dp(self.rb[0].view(np.float64)),
                              None if rb is None else _dp(self.rb[1].view(np.float64)), self.n_pol)

    def grid(self, i, k):
        """ln L^ML_{i k o t} [n_phi, n_t] (Eq. single_det_ML)."""
        NT = self.shape[4]
        out = np.zeros((self.n_phi, NT))
        if lib().or_presel_grid(ctypes.byref(self.s), ctypes.c_int64(i), int(k), _dp(out)):
            raise MemoryError("or_presel_grid")
        return out

    def run(self, delta=20.0, n_threads=0):
        """Every row: ml [I, D], arg_ot [I, D, 2], lnl_inco [I], keep [I], threshold, arg_i."""
        I, D = self.shape[:2]
        ml = np.zeros((I, D))
        arg = np.zeros((I, D, 2), dtype=np.int32)
        inco = np.zeros(I)
        keep = np.zeros(I, dtype=np.uint8)
        thr = ctypes.c_double(0.0)
        ai = ctypes.c_int64(0)
        if lib().or_presel(ctypes.byref(self.s), ctypes.c_double(delta), int(n_threads), _dp(ml),
                           arg.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(inco),
                           keep.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), ctypes.byref(thr),
                           ctypes.byref(ai)):
            raise MemoryError("or_presel")
        return dict(ml=ml, arg_ot=arg, lnl_inco=inco, keep=keep.astype(bool), threshold=thr.value,
                    arg_i=int(ai.value))


def rb_weights(f_fine, dff, psd, data, h0, nodes, t0=None):
    """Relative-binning weights (App. A, Eqs. dh_weights, hh_weights) with hat
    functions on the nodes f_fine[nodes], for the reference modes h0 [M, N]
    arriving at detector d at t0[d]: returns (w_dh [D, M, B], w_hh [D, M, M, B])."""
    f_fine = np.ascontiguousarray(f_fine, dtype=np.float64)
    dff = np.ascontiguousarray(dff, dtype=np.float64)
    psd = np.ascontiguousarray(psd, dtype=np.float64)
    data = _c128(data)
    h0 = _c128(h0)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    D, N = psd.shape
    M = h0.shape[0]
    B = nodes.shape[0]
    w_dh = np.zeros((D, M, B), np.complex128)
    w_hh = np.zeros((D, M, M, B), np.complex128)
    t0 = None if t0 is None else np.ascontiguousarray(t0, dtype=np.float64)
    if lib().or_rb_weights(D, M, ctypes.c_int64(N), _dp(f_fine), _dp(dff), _dp(psd), _dp(data.view(np.float64)),
                           _dp(h0.view(np.float64)), None if t0 is None else _dp(t0), B,
                           nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                           _dp(w_dh.view(np.float64)), _dp(w_hh.view(np.float64))):
        raise ValueError("reference waveform vanishes at a node")
    return w_dh, w_hh


def quad_ml(dh_p, dh_x, a, b, c):
    """Eqs. x_ML, single_det_ML for one (i, k, o, t)."""
    return lib().or_quad_ml(float(dh_p), float(dh_x), float(a), float(b), float(c))


def dist_marg(dh, hh, u_min):
    """Eq. lnl_dist_marginalized (pi(d_L) ~ d_L^2 up to d_max = d0/u_min)."""
    return lib().or_dist_marg(float(dh), float(hh), float(u_min))


def dist_sample(dh, hh, u_min, q):
    """Distance draw d_L / d_L^0 at cumulative probability q of the conditional
    density u^-4 exp(dh u - hh u^2/2), u = d_L^0/d_L >= u_min (App. C)."""
    return lib().or_dist_sample(float(dh), float(hh), float(u_min), float(q))


def posterior_samples(P, grid, ev, uniforms, threshold=-np.inf):
    """Resampling (Eq. posterior_element weights p_ieo = w_i w_e w_o Lbar_ieo):
    i from the row marginals, e from row i, o from the pair's phases (those that
    pass the ML cut at `threshold`), then the distance.  uniforms [n, 4]; the
    smallest index whose cumulative weight exceeds u * total is taken.
    Returns (i, e, o, d_L/d_L^0) arrays."""
    I, E = P.shape[:2]
    lw_e = P.ln_w_ext
    ln_pi = ev["ln_p_int"]

    def pick(lnw, u):
        m = np.max(lnw)
        c = np.cumsum(np.exp(lnw - m))
        return int(np.searchsorted(c, u * c[-1], side="right"))

    out_i, out_e, out_o, out_d = [], [], [], []
    for u1, u2, u3, u4 in np.asarray(uniforms, dtype=np.float64):
        i = pick(ln_pi, u1)
        e = pick(grid[i]["lnl_marg"] + lw_e, u2)
        z, H = P.mode_components(i, e)
        dh, hh = P.rotate_phases(z, H)
        lo = np.array([dist_marg(dh[o], hh[o], P.u_min) if lnl_ml(dh[o], hh[o]) >= threshold else -np.inf
                       for o in range(P.n_phi)])
        o = pick(lo, u3)
        out_i.append(i); out_e.append(e); out_o.append(o)
        out_d.append(dist_sample(dh[o], hh[o], P.u_min, u4))
    return np.array(out_i), np.array(out_e), np.array(out_o), np.array(out_d)


def lnl_ml(dh, hh):
    """Eq. bestfit_lnl."""
    return lib().or_lnl_ml(float(dh), float(hh))


def default_threads():
    return lib().or_default_threads()
