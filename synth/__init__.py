"""Seeded synthetic workloads for the dense (intrinsic x extrinsic) likelihood.

This module only *makes inputs*: a waveform bank on a compressed frequency
grid, a set of extrinsic samples (arrival times and complex detector
responses), a PSD per detector and one event's data (an injected bank member
plus Gaussian noise).  It contains none of the method's arithmetic (no inner
products, phase/distance marginalisation or evidence sums); both the FP64
oracle and the CUDA path consume what it returns.

Physical content, following the paper's decomposition (Sec. IV.A):

* waveform components h_m(f) = A_m f^(-7/6) exp(i Psi_m(f)) with the leading
  post-Newtonian phase Psi_22 and Psi_m = (m/2) Psi_22,
* detector responses F_+/F_x (Eqs. response_plus/response_cross) from the
  textbook detector-tensor contraction in an Earth-fixed frame,
* arrival times t_k = t_geo + r_k . n_prop / c (Eq. t_at_detector),
* the strain model h_k = u sum_m h_m R_{k,m} T_k Phi_m (Eq. h_k), used here
  only to build the injected signal.

The complex response R_{e,d,m} folds the polarisation sum of Eq. h_k into one
number per (extrinsic sample, detector, mode):
R = F_+ K+_m(iota) + F_x Kx_m(iota), with K+_m = (Y_lm + (-1)^l Y_l-m)/2 and
Kx_m = i (Y_lm - (-1)^l Y_l-m)/2 built from spin-weight -2 spherical
harmonics at azimuth 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Physical constants (SI).
C_LIGHT = 299_792_458.0
R_EARTH = 6.371e6
GM_SUN_S = 4.925491025543576e-06  # G M_sun / c^3 in seconds

# Approximate detector vertices (deg) and arm bearings (deg from North towards
# East).  Exact values are immaterial for a synthetic workload.
DETECTORS = {
    "H1": dict(lat=46.455, lon=-119.408, xarm=324.0, yarm=234.0),
    "L1": dict(lat=30.563, lon=-90.774, xarm=252.3, yarm=162.3),
    "V1": dict(lat=43.631, lon=10.504, xarm=70.6, yarm=340.6),
}
DET_ORDER = ("H1", "L1", "V1")
PSD_SCALES = (1.0, 1.3, 1.7)

# (l, m) for each supported mode count.  Modes are indexed by azimuthal m.
MODE_SETS = {
    1: ((2, 2),),
    2: ((2, 2), (3, 3)),
    3: ((2, 2), (3, 3), (4, 4)),
    4: ((2, 1), (2, 2), (3, 3), (4, 4)),
}


# ----------------------------------------------------------------------------
# frequency grid, quadrature weights, PSD
# ----------------------------------------------------------------------------
def freq_grid(n_bins: int, fmin: float = 20.0, fmax: float = 1024.0):
    """Log-spaced bins f_b and trapezoid weights w_b (Hz) on them."""
    f = fmin * (fmax / fmin) ** (np.arange(n_bins) / (n_bins - 1))
    w = np.empty(n_bins)
    w[0] = 0.5 * (f[1] - f[0])
    w[-1] = 0.5 * (f[-1] - f[-2])
    w[1:-1] = 0.5 * (f[2:] - f[:-2])
    return f, w


def analytic_psd(f: np.ndarray, scale: float = 1.0, f_s: float = 150.0):
    """Smooth analytic one-sided PSD in whitened units."""
    r = f / f_s
    return scale * (r ** -4 + 2.0 + 2.0 * r ** 2)


# ----------------------------------------------------------------------------
# spin-weight -2 spherical harmonics at azimuth 0 (real-valued there)
# ----------------------------------------------------------------------------
def sYlm_m2(l: int, m: int, iota):
    """_{-2}Y_{lm}(iota, phi=0) for the modes used here (closed forms)."""
    iota = np.asarray(iota, dtype=np.float64)
    c = np.cos(iota / 2.0)
    s = np.sin(iota / 2.0)
    ci = np.cos(iota)
    si = np.sin(iota)
    if l == 2 and m == 2:
        return math.sqrt(5.0 / (64.0 * math.pi)) * (1.0 + ci) ** 2
    if l == 2 and m == -2:
        return math.sqrt(5.0 / (64.0 * math.pi)) * (1.0 - ci) ** 2
    if l == 2 and m == 1:
        return math.sqrt(5.0 / (16.0 * math.pi)) * si * (1.0 + ci)
    if l == 2 and m == -1:
        return math.sqrt(5.0 / (16.0 * math.pi)) * si * (1.0 - ci)
    if l == 3 and m == 3:
        return -math.sqrt(21.0 / (2.0 * math.pi)) * c ** 5 * s
    if l == 3 and m == -3:
        return math.sqrt(21.0 / (2.0 * math.pi)) * c * s ** 5
    if l == 4 and m == 4:
        return 3.0 * math.sqrt(7.0 / math.pi) * c ** 6 * s ** 2
    if l == 4 and m == -4:
        return 3.0 * math.sqrt(7.0 / math.pi) * c ** 2 * s ** 6
    raise ValueError(f"no closed form for (l,m)=({l},{m})")


def polarisation_factors(l: int, m: int, iota):
    """(K+, Kx) such that h_+ = K+ h_lm and h_x = Kx h_lm for this mode."""
    yp = sYlm_m2(l, m, iota)
    ym = sYlm_m2(l, -m, iota)
    sign = (-1.0) ** l
    kplus = 0.5 * (yp + sign * ym)
    kcross = 0.5j * (yp - sign * ym)
    return kplus, kcross


# ----------------------------------------------------------------------------
# detector geometry (Earth-fixed frame; the sky rotates, the Earth does not)
# ----------------------------------------------------------------------------
def _unit(lat_deg, lon_deg):
    la, lo = math.radians(lat_deg), math.radians(lon_deg)
    return np.array([math.cos(la) * math.cos(lo), math.cos(la) * math.sin(lo), math.sin(la)])


def detector_geometry(name: str):
    """(position r [m], detector tensor D = (x x^T - y y^T)/2)."""
    g = DETECTORS[name]
    la, lo = math.radians(g["lat"]), math.radians(g["lon"])
    east = np.array([-math.sin(lo), math.cos(lo), 0.0])
    north = np.array([-math.sin(la) * math.cos(lo), -math.sin(la) * math.sin(lo), math.cos(la)])

    def arm(bearing_deg):
        b = math.radians(bearing_deg)
        return math.cos(b) * north + math.sin(b) * east

    x, y = arm(g["xarm"]), arm(g["yarm"])
    tensor = 0.5 * (np.outer(x, x) - np.outer(y, y))
    return R_EARTH * _unit(g["lat"], g["lon"]), tensor


def antenna_patterns(tensor, lat, lon, psi):
    """F_+, F_x for sources at Earth-fixed (lat, lon) with polarisation psi.

    Polarisation basis (X, Y) transverse to the source direction; F_+ = D:(XX-YY),
    F_x = D:(XY+YX).  Vectorised over the sample axis.
    """
    theta = 0.5 * np.pi - lat  # colatitude
    phi = lon
    sph, cph = np.sin(phi), np.cos(phi)
    sth, cth = np.sin(theta), np.cos(theta)
    sps, cps = np.sin(psi), np.cos(psi)
    X = np.stack([sph * cps - sps * cph * cth,
                  -(cph * cps + sps * sph * cth),
                  sps * sth], axis=-1)
    Y = np.stack([-sph * sps - cps * cph * cth,
                  cph * sps - cps * sph * cth,
                  cps * sth], axis=-1)
    fp = np.einsum("ni,ij,nj->n", X, tensor, X) - np.einsum("ni,ij,nj->n", Y, tensor, Y)
    fc = np.einsum("ni,ij,nj->n", X, tensor, Y) + np.einsum("ni,ij,nj->n", Y, tensor, X)
    return fp, fc


# ----------------------------------------------------------------------------
# workload containers
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Bank:
    f: np.ndarray          # [B] Hz
    w: np.ndarray          # [B] quadrature weights (Hz)
    mode_m: np.ndarray     # [M] azimuthal numbers
    mode_l: np.ndarray     # [M]
    h: np.ndarray          # [I, M, B] complex128
    ln_w: np.ndarray       # [I] ln(pi/pi') importance weights
    mchirp: np.ndarray     # [I] Msun (metadata)


@dataclasses.dataclass
class Extrinsic:
    t: np.ndarray          # [E, D] arrival time at each detector (s)
    R: np.ndarray          # [E, D, M] complex128 response
    ln_w: np.ndarray       # [E]
    lat: np.ndarray
    lon: np.ndarray
    psi: np.ndarray
    cos_iota: np.ndarray
    t_geo: np.ndarray
    F: np.ndarray = None   # [E, D, 2] real antenna patterns (F+, Fx), for polarisation-resolved banks


@dataclasses.dataclass
class Event:
    psd: np.ndarray        # [D, B]
    data: np.ndarray       # [D, B] complex128
    u_min: float           # d_L^0 / d_max of the distance prior
    n_phi: int
    injection: dict        # i, e (if inserted), phi, u, snr


# ----------------------------------------------------------------------------
# generators
# ----------------------------------------------------------------------------
def make_bank(rng, n_int, n_modes, n_bins, mc_range=(5.0, 30.0), ratio_max=0.3,
              ln_w="zero", dtype=np.complex128, fmin=20.0, fmax=1024.0,
              chunk=8192):
    """Leading-PN multi-mode bank on log-spaced bins (see module doc)."""
    f, w = freq_grid(n_bins, fmin, fmax)
    lm = MODE_SETS[n_modes]
    mode_l = np.array([l for l, _ in lm], dtype=np.int32)
    mode_m = np.array([m for _, m in lm], dtype=np.int32)
    mc = rng.uniform(mc_range[0], mc_range[1], size=n_int)
    ratios = rng.uniform(0.0, ratio_max, size=(n_int, n_modes))
    i22 = int(np.nonzero((mode_l == 2) & (mode_m == 2))[0][0])
    ratios[:, i22] = 1.0
    # normalise so that a waveform of chirp mass mc_ref has <h22|h22> = 1 on
    # the first detector's PSD with unit response
    psd0 = analytic_psd(f, PSD_SCALES[0])
    norm = math.sqrt(np.sum(4.0 * w * f ** (-7.0 / 3.0) / psd0))
    mc_ref = 0.5 * (mc_range[0] + mc_range[1])
    amp22 = (mc / mc_ref) ** (5.0 / 6.0) / norm
    h = np.empty((n_int, n_modes, n_bins), dtype=dtype)
    base_amp = f ** (-7.0 / 6.0)
    for i0 in range(0, n_int, chunk):
        i1 = min(n_int, i0 + chunk)
        x = np.pi * GM_SUN_S * mc[i0:i1, None] * f[None, :]
        psi22 = -0.25 * np.pi + (3.0 / 128.0) * x ** (-5.0 / 3.0)
        for k, m in enumerate(mode_m):
            amp = (amp22[i0:i1] * ratios[i0:i1, k])[:, None] * base_amp[None, :]
            h[i0:i1, k, :] = amp * np.exp(1j * (0.5 * m) * psi22)
    if ln_w == "zero":
        lw = np.zeros(n_int)
    elif ln_w == "random":
        lw = rng.normal(0.0, 0.5, size=n_int)
    else:
        raise ValueError(ln_w)
    return Bank(f=f, w=w, mode_m=mode_m, mode_l=mode_l, h=h, ln_w=lw, mchirp=mc)


def make_extrinsic(rng, n_ext, n_det, bank: Bank, ln_w="zero", t_span=0.010):
    """Prior draws: isotropic sky, uniform psi, cos(iota), t_geo in +-t_span."""
    lon = rng.uniform(0.0, 2.0 * np.pi, n_ext)
    lat = np.arcsin(rng.uniform(-1.0, 1.0, n_ext))
    psi = rng.uniform(0.0, np.pi, n_ext)
    cos_iota = rng.uniform(-1.0, 1.0, n_ext)
    t_geo = rng.uniform(-t_span, t_span, n_ext)
    return extrinsic_from_params(lat, lon, psi, cos_iota, t_geo, n_det, bank,
                                 ln_w=(np.zeros(n_ext) if ln_w == "zero"
                                       else rng.normal(0.0, 0.5, n_ext)))


def extrinsic_from_params(lat, lon, psi, cos_iota, t_geo, n_det, bank: Bank, ln_w):
    n_ext = lat.shape[0]
    iota = np.arccos(cos_iota)
    # propagation direction is minus the source direction
    n_src = np.stack([np.cos(lat) * np.cos(lon), np.cos(lat) * np.sin(lon), np.sin(lat)], -1)
    M = bank.mode_m.shape[0]
    t = np.empty((n_ext, n_det))
    R = np.empty((n_ext, n_det, M), dtype=np.complex128)
    kp = np.empty((n_ext, M), dtype=np.complex128)
    kx = np.empty((n_ext, M), dtype=np.complex128)
    for k in range(M):
        a, b = polarisation_factors(int(bank.mode_l[k]), int(bank.mode_m[k]), iota)
        kp[:, k] = a
        kx[:, k] = b
    for d in range(n_det):
        r, tensor = detector_geometry(DET_ORDER[d])
        t[:, d] = t_geo - (n_src @ r) / C_LIGHT
        fp, fc = antenna_patterns(tensor, lat, lon, psi)
        R[:, d, :] = fp[:, None] * kp + fc[:, None] * kx
    F = np.empty((n_ext, n_det, 2))
    for d in range(n_det):
        _, tensor = detector_geometry(DET_ORDER[d])
        F[:, d, 0], F[:, d, 1] = antenna_patterns(tensor, lat, lon, psi)
    return Extrinsic(t=t, R=R, ln_w=np.asarray(ln_w, dtype=np.float64), lat=lat, lon=lon,
                     psi=psi, cos_iota=cos_iota, t_geo=t_geo, F=F)


def signal_at_detectors(h_modes, R_dm, t_d, f, mode_m, phi, u):
    """Eq. h_k: u sum_m h_m R_{d,m} exp(-2 pi i f t_d) exp(i m phi); [D, B]."""
    ph = np.exp(1j * mode_m * phi)                      # [M]
    shift = np.exp(-2j * np.pi * f[None, :] * t_d[:, None])   # [D, B]
    comb = np.einsum("mb,dm,m->db", h_modes, R_dm, ph)
    return u * comb * shift


def network_norm(sig, psd, w):
    """sum_d sum_b 4 w |s|^2 / S  (only used to scale the injection)."""
    return float(np.sum(4.0 * w[None, :] * np.abs(sig) ** 2 / psd))


def make_event(rng, bank: Bank, ext: Extrinsic, n_det, snr=15.0, n_phi=32,
               noise=True, inj_i=None, inj_e=None, phi_inj=None, u_min=None):
    """Event data: bank member inj_i seen through extrinsic sample inj_e.

    If inj_e is None a fresh prior draw is used (not a member of `ext`).
    The distance is set so that the network optimal SNR equals `snr`.
    """
    D = n_det
    psd = np.stack([analytic_psd(bank.f, PSD_SCALES[d]) for d in range(D)])
    I = bank.h.shape[0]
    if inj_i is None:
        inj_i = int(rng.integers(0, I))
    if inj_e is None:
        e1 = make_extrinsic(rng, 1, D, bank)
        R_dm, t_d, cos_iota = e1.R[0], e1.t[0], float(e1.cos_iota[0])
    else:
        R_dm, t_d, cos_iota = ext.R[inj_e], ext.t[inj_e], float(ext.cos_iota[inj_e])
    if phi_inj is None:
        phi_inj = float(rng.uniform(0.0, 2.0 * np.pi))
    h_modes = np.asarray(bank.h[inj_i], dtype=np.complex128)
    unit = signal_at_detectors(h_modes, R_dm, t_d, bank.f, bank.mode_m, phi_inj, 1.0)
    u_inj = snr / math.sqrt(network_norm(unit, psd, bank.w))
    data = u_inj * unit
    if noise:
        sigma = np.sqrt(psd / (4.0 * bank.w[None, :]))
        data = data + sigma * (rng.standard_normal((D, bank.f.size))
                               + 1j * rng.standard_normal((D, bank.f.size)))
    if u_min is None:
        u_min = default_u_min(bank, D)
    return Event(psd=psd, data=data, u_min=float(u_min), n_phi=int(n_phi),
                 injection=dict(i=inj_i, e=inj_e, phi=phi_inj, u=u_inj, snr=snr,
                                cos_iota=cos_iota, t_det=np.array(t_d, dtype=np.float64)))


def default_u_min(bank: Bank, n_det: int, snr_at_dmax: float = 4.0):
    """u_min = d0/d_max such that a face-on, optimally oriented waveform of
    <h22|h22> = 1 reaches network SNR `snr_at_dmax` at d_max."""
    kp, _ = polarisation_factors(2, 2, 0.0)
    rho2 = sum(abs(kp) ** 2 / PSD_SCALES[d] for d in range(n_det))
    return snr_at_dmax / math.sqrt(rho2)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
WORKLOADS = {
    # name: (I, E, D, M, B, snr, seed)
    "cfg1": dict(n_int=1024, n_ext=256, n_det=2, n_modes=3, n_bins=256, snr=15.0, seed=0),
    "cfg2": dict(n_int=65536, n_ext=4096, n_det=3, n_modes=4, n_bins=512, snr=15.0, seed=2),
    "cfg3": dict(n_int=1048576, n_ext=2048, n_det=3, n_modes=4, n_bins=384, snr=30.0, seed=3),
}


@dataclasses.dataclass
class Workload:
    bank: Bank
    ext: Extrinsic
    event: Event


def make_workload(n_int, n_ext, n_det, n_modes, n_bins, snr=15.0, seed=0, n_phi=32,
                  noise=True, insert_injection=False, ln_w="zero", bank_dtype=np.complex128,
                  phi_inj=None):
    """Bank + extrinsic set + one event, all from one seeded generator.

    insert_injection=True places the injected extrinsic sample at e = 0 (and,
    unless phi_inj is given, the injected phase at phi = 0) so that the
    noiseless likelihood peaks exactly on the grid.
    """
    rng = np.random.default_rng(seed)
    bank = make_bank(rng, n_int, n_modes, n_bins, ln_w=ln_w, dtype=bank_dtype)
    ext = make_extrinsic(rng, n_ext, n_det, bank, ln_w=ln_w)
    if insert_injection:
        ev = make_event(rng, bank, ext, n_det, snr=snr, n_phi=n_phi, noise=noise,
                        inj_e=0, phi_inj=(0.0 if phi_inj is None else phi_inj))
    else:
        ev = make_event(rng, bank, ext, n_det, snr=snr, n_phi=n_phi, noise=noise,
                        phi_inj=phi_inj)
    return Workload(bank=bank, ext=ext, event=ev)


@dataclasses.dataclass
class BatchWorkload:
    bank: Bank
    events: list  # [(Extrinsic, Event)]


def make_batch_workload(n_events=64, n_int=262144, n_modes=4, n_bins=512, seed=4,
                        e_choices=(512, 1024, 2048, 4096), d_choices=(2, 3), snr_range=(8.0, 40.0),
                        bank_dtype=np.complex128):
    """Many events over one shared bank: per event an extrinsic count drawn from
    e_choices, a detector count from d_choices and an injection SNR uniform in
    snr_range (prior-drawn extrinsic samples, a random bank member injected)."""
    rng = np.random.default_rng(seed)
    bank = make_bank(rng, n_int, n_modes, n_bins, dtype=bank_dtype)
    events = []
    for _ in range(n_events):
        E = int(rng.choice(e_choices))
        D = int(rng.choice(d_choices))
        snr = float(rng.uniform(*snr_range))
        ext = make_extrinsic(rng, E, D, bank)
        events.append((ext, make_event(rng, bank, ext, D, snr=snr)))
    return BatchWorkload(bank=bank, events=events)


@dataclasses.dataclass
class Arrival:
    t: float            # arrival time (s) from the start of the stream
    n_bins: int         # which bank (one per bin grid)
    i0: int
    i1: int             # bank slice [i0, i1)
    ext: Extrinsic
    event: Event


def make_serving_stream(n_events=2000, rate=20.0, seed=5, n_int=524288, n_modes=4, bins=(256, 512),
                        slice_range=(16384, 524288), e_range=(1024, 8192), d_choices=(2, 3),
                        snr_range=(8.0, 50.0), pool=8, bank_dtype=np.complex64):
    """A Poisson stream of events (exponential inter-arrival times of mean
    1/rate) against resident banks, one per bin grid in `bins`.  Per event: a
    bin grid, a bank slice of uniform length in slice_range at a uniform
    offset, an extrinsic count uniform in e_range (the first E samples of one
    of `pool` prior-drawn sets per detector count), a detector count and an
    injection SNR uniform in snr_range, the injected member inside the slice."""
    rng = np.random.default_rng(seed)
    banks = {B: make_bank(rng, n_int, n_modes, B, dtype=bank_dtype) for B in bins}
    emax = e_range[1]
    pools = {(B, D): [make_extrinsic(rng, emax, D, banks[B]) for _ in range(pool)]
             for B in bins for D in d_choices}
    t = 0.0
    stream = []
    for _ in range(n_events):
        t += float(rng.exponential(1.0 / rate))
        B = int(rng.choice(bins))
        D = int(rng.choice(d_choices))
        L = int(rng.integers(slice_range[0], slice_range[1] + 1))
        i0 = int(rng.integers(0, n_int - L + 1))
        E = int(rng.integers(e_range[0], e_range[1] + 1))
        src = pools[(B, D)][int(rng.integers(0, pool))]
        ext = Extrinsic(t=src.t[:E], R=src.R[:E], ln_w=src.ln_w[:E], lat=src.lat[:E], lon=src.lon[:E],
                        psi=src.psi[:E], cos_iota=src.cos_iota[:E], t_geo=src.t_geo[:E])
        ev = make_event(rng, banks[B], ext, D, snr=float(rng.uniform(*snr_range)),
                        inj_i=int(rng.integers(i0, i0 + L)))
        stream.append(Arrival(t=t, n_bins=B, i0=i0, i1=i0 + L, ext=ext, event=ev))
    return banks, stream


@dataclasses.dataclass
class PreselInputs:
    """Inputs of the incoherent single-detector pre-selection (Sec. IV.D, App. B)."""
    pol: np.ndarray        # [I, M, 2] complex128: K_{i m +}, K_{i m x}
    cos_iota: np.ndarray   # [I] inclination of each bank row (an intrinsic parameter there)
    t_grid: np.ndarray     # [D, n_t] arrival-time grid at each detector (s)


def row_polarisation_factors(bank: Bank, cos_iota):
    """K_{i m p} of every row: h_{i m p} = K_{i m p} h_{i m} (App. B's h_impb)."""
    iota = np.arccos(np.asarray(cos_iota, dtype=np.float64))
    M = bank.mode_m.shape[0]
    pol = np.empty((iota.shape[0], M, 2), dtype=np.complex128)
    for k in range(M):
        a, b = polarisation_factors(int(bank.mode_l[k]), int(bank.mode_m[k]), iota)
        pol[:, k, 0] = a
        pol[:, k, 1] = b
    return pol


def make_presel_inputs(wl: "Workload", n_t=128, dt=5.0e-4, seed=7):
    """Rows draw cos(iota) ~ U[-1, 1] (the bank's inclination prior); the
    injected row takes the injection's.  The time grid is shared by the
    detectors: n_t points spaced dt, centred on the geocentric trigger time 0,
    so it spans the prior's t_geo window plus the light travel time across
    the Earth (n_t dt = 64 ms at the defaults)."""
    rng = np.random.default_rng(seed)
    I = wl.bank.h.shape[0]
    cos_iota = rng.uniform(-1.0, 1.0, I)
    inj = wl.event.injection
    if inj.get("cos_iota") is not None and 0 <= inj["i"] < I:
        cos_iota[inj["i"]] = inj["cos_iota"]
    D = wl.event.psd.shape[0]
    t = (np.arange(n_t) - n_t // 2) * dt
    return PreselInputs(pol=row_polarisation_factors(wl.bank, cos_iota), cos_iota=cos_iota,
                        t_grid=np.tile(t, (D, 1)))


# ----------------------------------------------------------------------------
# relative binning (App. A): full-resolution data, a reference waveform, a bank
# stored on coarse nodes of the fine grid
# ----------------------------------------------------------------------------
def waveform_modes(f, mc, ratios, mode_m, amp22):
    """The bank's waveform model (module doc) for rows (mc [n], ratios [n, M],
    amp22 [n]) on any frequencies f: complex [n, M, len(f)]."""
    mc = np.atleast_1d(np.asarray(mc, dtype=np.float64))
    x = np.pi * GM_SUN_S * mc[:, None] * f[None, :]
    psi22 = -0.25 * np.pi + (3.0 / 128.0) * x ** (-5.0 / 3.0)
    base = f ** (-7.0 / 6.0)
    out = np.empty((mc.shape[0], len(mode_m), f.shape[0]), dtype=np.complex128)
    for k, m in enumerate(mode_m):
        out[:, k, :] = (amp22 * ratios[:, k])[:, None] * base[None, :] * np.exp(1j * (0.5 * m) * psi22)
    return out


@dataclasses.dataclass
class RBWorkload:
    bank: Bank             # rows on the coarse nodes f_fine[nodes]; row 0 is the reference
    ext: Extrinsic
    event: Event           # psd and data sampled at the nodes (plain quadrature on the same bins)
    f_fine: np.ndarray     # [N] uniform grid (Hz)
    dff: np.ndarray        # [N] trapezoid weights (Hz)
    psd_fine: np.ndarray   # [D, N]
    data_fine: np.ndarray  # [D, N] complex
    h0_fine: np.ndarray    # [J, N] complex: the reference waveform's components (modes, or
                           # (mode, polarisation) pairs j = 2m + p of a polarisation-resolved bank)
    t0: np.ndarray         # [D] the reference's arrival time at each detector (s)
    nodes: np.ndarray      # [B] increasing indices into f_fine
    ratios: np.ndarray     # [I, M] mode amplitude ratios of the rows
    amp22: np.ndarray      # [I] 22-mode amplitude scale of the rows
    wobble: tuple = None   # (iota0, amp, per) per row of a polarisation-resolved bank, else None

    def rows_fine(self, rows):
        """The bank rows on the fine grid: complex [len(rows), M, N], or
        [len(rows), M, 2, N] for a polarisation-resolved bank."""
        rows = np.atleast_1d(rows)
        h = waveform_modes(self.f_fine, self.bank.mchirp[rows], self.ratios[rows], self.bank.mode_m,
                           self.amp22[rows])
        if self.wobble is None:
            return h
        iota0, amp, per = (x[rows] for x in self.wobble)
        return wobbled_polarisations(h, self.f_fine, self.bank.mode_l, self.bank.mode_m, iota0, amp, per,
                                     self.f_fine[0])


def make_rb_workload(n_int, n_ext, n_det, n_modes, n_bins, n_fine=65536, snr=15.0, seed=0, mc0=12.0,
                     spread=0.02, n_phi=32, noise=True, sky_sigma=0.05, t_sigma=5e-4, fmin=20.0, fmax=1024.0,
                     precessing=False):
    """Full-resolution event and a bank stored on coarse nodes (App. A).

    The fine grid is uniform over [fmin, fmax] with n_fine points; the nodes are
    the fine points nearest to n_bins log-spaced frequencies.  The reference
    waveform (row 0 of the bank, chirp mass mc0, mode ratios in [0.05, 0.3]) is
    also the injection; the other rows have chirp masses within +-spread of
    mc0 (a bank around the signal, as the pre-selection leaves it) and mode
    ratios U[0, 0.3].  Extrinsic samples concentrate near the injection (sky
    offsets N(0, sky_sigma) rad, arrival offsets N(0, t_sigma) s, psi and
    cos(iota) from the prior), like the output of an adaptive extrinsic
    sampler, so that the time shifts relative to the reference stay small.
    The reference's arrival times t0 are the injection's.
    precessing: a polarisation-resolved bank h_{imp} (each row's inclination
    wobbling with frequency as in precessing_bank, the reference's too), data
    sum_{m,p} F_dp h0_mp e^{i m phi} T_d, and h0_fine the reference's 2M
    components j = 2m + p, so that the weights carry the polarisation index of
    App. A (W_{kmpb}, W_{kmm'pp'b}).
    """
    rng = np.random.default_rng(seed)
    f_fine = np.linspace(fmin, fmax, n_fine)
    dff = np.full(n_fine, f_fine[1] - f_fine[0])
    dff[0] *= 0.5
    dff[-1] *= 0.5
    target = fmin * (fmax / fmin) ** (np.arange(n_bins) / (n_bins - 1))
    nodes = np.unique(np.clip(np.rint((target - fmin) / (f_fine[1] - f_fine[0])).astype(np.int64), 0, n_fine - 1))
    if nodes.shape[0] != n_bins:
        raise ValueError("fine grid too coarse for the requested nodes")
    fb = f_fine[nodes]
    lm = MODE_SETS[n_modes]
    mode_l = np.array([l for l, _ in lm], dtype=np.int32)
    mode_m = np.array([m for _, m in lm], dtype=np.int32)
    i22 = int(np.nonzero((mode_l == 2) & (mode_m == 2))[0][0])
    mc = mc0 * (1.0 + rng.uniform(-spread, spread, n_int))
    mc[0] = mc0
    ratios = rng.uniform(0.0, 0.3, (n_int, n_modes))
    ratios[0] = rng.uniform(0.05, 0.3, n_modes)
    ratios[:, i22] = 1.0
    psd_fine = np.stack([analytic_psd(f_fine, PSD_SCALES[d]) for d in range(n_det)])
    norm = math.sqrt(np.sum(4.0 * dff * f_fine ** (-7.0 / 3.0) / psd_fine[0]))
    amp22 = (mc / mc0) ** (5.0 / 6.0) / norm
    h = waveform_modes(fb, mc, ratios, mode_m, amp22)
    wob = None
    if precessing:
        wob = (np.arccos(rng.uniform(-1.0, 1.0, n_int)), rng.uniform(0.0, 0.5, n_int), rng.uniform(0.5, 2.0, n_int))
        h = wobbled_polarisations(h, fb, mode_l, mode_m, *wob, fmin)
    # coarse-grid quadrature weights for the plain comparison on the same bins
    w = np.empty(n_bins)
    w[0] = 0.5 * (fb[1] - fb[0])
    w[-1] = 0.5 * (fb[-1] - fb[-2])
    w[1:-1] = 0.5 * (fb[2:] - fb[:-2])
    bank = Bank(f=fb, w=w, mode_m=mode_m, mode_l=mode_l, h=h, ln_w=np.zeros(n_int), mchirp=mc)
    # injection: the reference through a prior draw at a random phase
    e1 = make_extrinsic(rng, 1, n_det, bank)
    phi_inj = float(rng.uniform(0.0, 2.0 * np.pi))
    h0 = waveform_modes(f_fine, mc[:1], ratios[:1], mode_m, amp22[:1])[0]
    if precessing:
        h0p = wobbled_polarisations(h0[None], f_fine, mode_l, mode_m, *(x[:1] for x in wob), fmin)[0]  # [M, 2, N]
        ph = np.exp(1j * mode_m * phi_inj)
        shift = np.exp(-2j * np.pi * f_fine[None, :] * e1.t[0][:, None])
        unit = np.einsum("mpn,dp,m->dn", h0p, e1.F[0], ph) * shift
        h0 = h0p.reshape(2 * n_modes, n_fine)
    else:
        unit = signal_at_detectors(h0, e1.R[0], e1.t[0], f_fine, mode_m, phi_inj, 1.0)
    u_inj = snr / math.sqrt(float(np.sum(4.0 * dff[None, :] * np.abs(unit) ** 2 / psd_fine)))
    data_fine = u_inj * unit
    if noise:
        sigma = np.sqrt(psd_fine / (4.0 * dff[None, :]))
        data_fine = data_fine + sigma * (rng.standard_normal(sigma.shape) + 1j * rng.standard_normal(sigma.shape))
    # extrinsic samples near the injection
    lat = np.clip(e1.lat[0] + rng.normal(0.0, sky_sigma, n_ext), -0.5 * np.pi, 0.5 * np.pi)
    lon = e1.lon[0] + rng.normal(0.0, sky_sigma, n_ext)
    psi = rng.uniform(0.0, np.pi, n_ext)
    cos_iota = rng.uniform(-1.0, 1.0, n_ext)
    t_geo = e1.t_geo[0] + rng.normal(0.0, t_sigma, n_ext)
    ext = extrinsic_from_params(lat, lon, psi, cos_iota, t_geo, n_det, bank, ln_w=np.zeros(n_ext))
    ev = Event(psd=psd_fine[:, nodes].copy(), data=data_fine[:, nodes].copy(), u_min=default_u_min(bank, n_det),
               n_phi=int(n_phi), injection=dict(i=0, e=None, phi=phi_inj, u=u_inj, snr=snr,
                                                cos_iota=float(e1.cos_iota[0]), t_det=e1.t[0].copy()))
    return RBWorkload(bank=bank, ext=ext, event=ev, f_fine=f_fine, dff=dff, psd_fine=psd_fine, data_fine=data_fine,
                      h0_fine=h0, t0=e1.t[0].copy(), nodes=nodes, ratios=ratios, amp22=amp22, wobble=wob)


# ----------------------------------------------------------------------------
# polarisation-resolved (precessing) banks: h_{i m p}(f), p = +, x
# ----------------------------------------------------------------------------
def wobbled_polarisations(h, f, mode_l, mode_m, iota0, amp, per, f0):
    """h_{i m p}(f) = K_{m p}(iota_i(f)) h_{i m}(f) with iota_i(f) = iota0_i +
    amp_i sin(2 pi ln(f/f0) / per_i): h [I, M, N] -> [I, M, 2, N]."""
    I, M, N = h.shape
    x = np.log(f / f0)
    iota = iota0[:, None] + amp[:, None] * np.sin(2.0 * np.pi * x[None, :] / per[:, None])
    out = np.empty((I, M, 2, N), dtype=np.complex128)
    for k in range(M):
        kp, kx = polarisation_factors(int(mode_l[k]), int(mode_m[k]), iota)
        out[:, k, 0, :] = kp * h[:, k, :]
        out[:, k, 1, :] = kx * h[:, k, :]
    return out


def precessing_bank(base: Bank, rng, wobble_max=0.5):
    """A polarisation-resolved bank from a non-precessing one: each row's
    inclination wobbles with frequency, iota_i(f) = iota0_i + a_i sin(2 pi
    ln(f/f_0) / L_i) (a_i ~ U[0, wobble_max] rad, L_i ~ U[0.5, 2], cos iota0 ~
    U[-1, 1]), standing in for the spin-precession of the paper's general case
    (Sec. IV.A): h_{i m p}(f) = K_{m p}(iota_i(f)) h_{i m}(f), whose + / x ratio
    is not fixed per mode.  Returns h [I, M, 2, B] and iota0 [I]."""
    I = base.h.shape[0]
    iota0 = np.arccos(rng.uniform(-1.0, 1.0, I))
    amp = rng.uniform(0.0, wobble_max, I)
    per = rng.uniform(0.5, 2.0, I)
    return wobbled_polarisations(base.h, base.f, base.mode_l, base.mode_m, iota0, amp, per, base.f[0]), iota0


def make_precessing_workload(n_int, n_ext, n_det, n_modes, n_bins, snr=15.0, seed=0, n_phi=32, noise=True,
                             insert_injection=False, ln_w="zero"):
    """Bank (polarisation-resolved), extrinsic samples (with F) and one event
    whose signal is sum_{m,p} F_{dp} h_{i* m p} e^{i m phi} T_d (Eq. h_k with the
    polarisation index), scaled to network SNR `snr`, plus noise.
    insert_injection: the injected sample is extrinsic sample 0 at phase 0."""
    rng = np.random.default_rng(seed)
    base = make_bank(rng, n_int, n_modes, n_bins, ln_w=ln_w)
    hp, _ = precessing_bank(base, rng)
    bank = Bank(f=base.f, w=base.w, mode_m=base.mode_m, mode_l=base.mode_l, h=hp, ln_w=base.ln_w,
                mchirp=base.mchirp)
    ext = make_extrinsic(rng, n_ext, n_det, base, ln_w=ln_w)
    psd = np.stack([analytic_psd(bank.f, PSD_SCALES[d]) for d in range(n_det)])
    inj_i = int(rng.integers(0, n_int))
    if insert_injection:
        Fd, td, phi = ext.F[0], ext.t[0], 0.0
    else:
        e1 = make_extrinsic(rng, 1, n_det, base)
        Fd, td, phi = e1.F[0], e1.t[0], float(rng.uniform(0.0, 2.0 * np.pi))
    ph = np.exp(1j * bank.mode_m * phi)
    shift = np.exp(-2j * np.pi * bank.f[None, :] * td[:, None])
    unit = np.einsum("mpb,dp,m->db", hp[inj_i], Fd, ph) * shift
    u_inj = snr / math.sqrt(network_norm(unit, psd, bank.w))
    data = u_inj * unit
    if noise:
        sigma = np.sqrt(psd / (4.0 * bank.w[None, :]))
        data = data + sigma * (rng.standard_normal(sigma.shape) + 1j * rng.standard_normal(sigma.shape))
    ev = Event(psd=psd, data=data, u_min=default_u_min(base, n_det), n_phi=int(n_phi),
               injection=dict(i=inj_i, e=0 if insert_injection else None, phi=phi, u=u_inj, snr=snr,
                              cos_iota=None, t_det=np.array(td)))
    return Workload(bank=bank, ext=ext, event=ev)


def named_workload(name: str, **overrides):
    kw = dict(WORKLOADS[name])
    kw.update(overrides)
    return make_workload(**kw)


def pair_subsample(rng_seed, n_int, n_ext, frac=0.01, n_max=None):
    """Seeded uniform (i, e) subsample without replacement, sorted."""
    rng = np.random.default_rng(rng_seed)
    n = n_int * n_ext
    k = max(1, int(round(frac * n)))
    if n_max is not None:
        k = min(k, n_max)
    flat = np.sort(rng.choice(n, size=k, replace=False))
    return (flat // n_ext).astype(np.int64), (flat % n_ext).astype(np.int64)
