"""Pins of the FP64 oracle against what the mathematics fixes.

None of these re-types an oracle formula: each compares the oracle with a
closed form, an independent quadrature, a textbook special function, an
identity computed by a different formula, a hand-evaluated case, brute force
in plain Python on tiny inputs, or sampling statistics.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import synth


# ---------------------------------------------------------------------------
# Eq. lnl_dist_marginalized
# ---------------------------------------------------------------------------
def _closed_form_dh0(hh, u_min):
    # int_0^dmax 3 d^2/dmax^3 exp(-hh (d0/d)^2 / 2) dd, by parts (a = sqrt(hh) u_min):
    # e^{-a^2/2} - a^2 [e^{-a^2/2} - sqrt(pi/2) a erfc(a/sqrt 2)]
    a = math.sqrt(hh) * u_min
    return math.exp(-a * a / 2) - a * a * (math.exp(-a * a / 2)
                                           - math.sqrt(math.pi / 2) * a * math.erfc(a / math.sqrt(2)))


@pytest.mark.parametrize("hh,u_min", [(0.5, 2.0), (1.0, 1.0), (4.0, 0.3), (0.02, 9.5),
                                      (3.0, 2.5), (1e-4, 1.0)])
def test_dist_marg_closed_form_at_zero_dh(oracle_lib, hh, u_min):
    got = oracle_lib.dist_marg(0.0, hh, u_min)
    assert got == pytest.approx(math.log(_closed_form_dh0(hh, u_min)), abs=1e-11)


@pytest.mark.parametrize("dh,hh,u_min", [(10.0, 1.0, 2.0), (-3.0, 2.0, 1.0), (50.0, 20.0, 0.5),
                                         (0.1, 0.01, 3.0), (1.7, 0.013, 9.5), (0.6, 0.02, 9.5),
                                         (-0.2, 0.05, 9.5), (30.0, 4.0, 0.1)])
def test_dist_marg_vs_quadrature_in_distance(oracle_lib, dh, hh, u_min):
    # the untransformed integral over d_L with pi(d_L) = 3 d^2 / dmax^3, d0 = 1
    dmax = 1.0 / u_min
    f = lambda d: 3 * d * d / dmax ** 3 * math.exp(dh / d - 0.5 * hh / d ** 2)
    pts = [hh / dh] if (dh > 0 and hh / dh < dmax) else None
    val, _ = integrate.quad(f, 0.0, dmax, points=pts, limit=500, epsabs=0, epsrel=1e-12)
    assert oracle_lib.dist_marg(dh, hh, u_min) == pytest.approx(math.log(val), abs=1e-9)


@pytest.mark.parametrize("x,s", [(100.0, 1.0), (120.0, 3.0), (80.0, 0.5)])
def test_dist_marg_laplace_asymptote(oracle_lib, x, s):
    # x = dh/sqrt(hh) >> s: ln Lbar -> x^2/2 + ln(3 s^3 sqrt(2 pi)) - 4 ln x
    #                                  + ln(1 + 10/x^2 + 105/x^4) + O(x^-6)
    hh = 2.0
    dh, u_min = x * math.sqrt(hh), s / math.sqrt(hh)
    expect = (0.5 * x * x + math.log(3 * s ** 3 * math.sqrt(2 * math.pi)) - 4 * math.log(x)
              + math.log1p(10 / x ** 2 + 105 / x ** 4))
    assert oracle_lib.dist_marg(dh, hh, u_min) == pytest.approx(expect, abs=2e-8)


def test_dist_marg_limits_and_monotonicity(oracle_lib):
    # no signal power -> likelihood ratio 1; small power -> ln Lbar -> 0
    assert oracle_lib.dist_marg(0.3, 0.0, 2.0) == 0.0
    assert abs(oracle_lib.dist_marg(1e-5, 1e-10, 2.0)) < 1e-4
    # monotone increasing in dh at fixed hh
    vals = [oracle_lib.dist_marg(dh, 1.5, 1.2) for dh in np.linspace(-20, 40, 61)]
    assert np.all(np.diff(vals) > 0)
    # Lbar <= exp(ln L^ML) since the prior integrates to one
    for dh, hh in [(3.0, 1.0), (30.0, 5.0), (-2.0, 1.0), (1.7, 0.013)]:
        assert oracle_lib.dist_marg(dh, hh, 9.5) <= oracle_lib.lnl_ml(dh, hh) + 1e-12


# ---------------------------------------------------------------------------
# Eq. bestfit_lnl
# ---------------------------------------------------------------------------
def test_lnl_ml_is_max_over_distance(oracle_lib):
    for dh, hh in [(3.0, 1.0), (0.5, 2.0), (-1.0, 1.0), (40.0, 7.0)]:
        u = np.linspace(0, 100, 200001)
        brute = max(0.0, float(np.max(dh * u - 0.5 * hh * u * u)))
        assert oracle_lib.lnl_ml(dh, hh) == pytest.approx(brute, abs=1e-6)


# ---------------------------------------------------------------------------
# hand-evaluated tiny case: one bin, one detector, one mode m = 2
# ---------------------------------------------------------------------------
def _tiny_problem(oracle_lib, n_phi=4, t=0.0, R=1.0 + 0.0j, d=1.0 + 0.0j, h=1.0 + 0.0j):
    bank = synth.Bank(f=np.array([1.0]), w=np.array([1.0]), mode_m=np.array([2], np.int32),
                      mode_l=np.array([2], np.int32), h=np.array([[[h]]], np.complex128),
                      ln_w=np.zeros(1), mchirp=np.zeros(1))
    ext = synth.Extrinsic(t=np.array([[t]]), R=np.array([[[R]]], np.complex128), ln_w=np.zeros(1),
                          lat=None, lon=None, psi=None, cos_iota=None, t_geo=None)
    ev = synth.Event(psd=np.array([[4.0]]), data=np.array([[d]], np.complex128), u_min=1.0,
                     n_phi=n_phi, injection={})
    return oracle_lib.OracleProblem(bank, ext, ev)


def test_tiny_hand_evaluated(oracle_lib):
    # 4 w / S = 1;  h_d = h R e^{2 i phi} e^{-2 pi i f t};  <d|h> = d conj(h_d)
    P = _tiny_problem(oracle_lib)
    for route in ("O1", "O2"):
        if route == "O1":
            dh, hh = P.direct_phases(0, 0)
        else:
            z, H = P.mode_components(0, 0)
            dh, hh = P.rotate_phases(z, H)
        # phi_o = 0, pi/2, pi, 3pi/2 -> Re e^{-2 i phi} = 1, -1, 1, -1
        np.testing.assert_allclose(dh, [1, -1, 1, -1], atol=1e-15)
        np.testing.assert_allclose(hh, [1, 1, 1, 1], atol=1e-15)
    assert [oracle_lib.lnl_ml(a, b) for a, b in zip(dh, hh)] == [0.5, 0.0, 0.5, 0.0]
    # a quarter-cycle time shift at f = 1 Hz (t = 1/4 s) rotates <d|h> by +i:
    # Re(d conj(h e^{-i pi/2} e^{2 i phi})) = Re(i e^{-2 i phi}) = sin(2 phi)
    P = _tiny_problem(oracle_lib, n_phi=8, t=0.25)
    dh, hh = P.direct_phases(0, 0)
    phi = 2 * np.pi * np.arange(8) / 8
    np.testing.assert_allclose(dh, np.sin(2 * phi), atol=1e-14)
    # complex response R = 2i: |R|^2 = 4 scales <h|h>, phase -pi/2 enters <d|h>
    P = _tiny_problem(oracle_lib, n_phi=4, R=2j)
    dh, hh = P.direct_phases(0, 0)
    np.testing.assert_allclose(hh, [4, 4, 4, 4], atol=1e-14)
    # Re(conj(2 i e^{2 i phi})) = Re(-2 i e^{-2 i phi}) = -2 sin(2 phi) = 0 on this grid
    np.testing.assert_allclose(dh, [0, 0, 0, 0], atol=1e-14)


# ---------------------------------------------------------------------------
# route O1 (direct) vs route O2 (components); invariants
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_noisy(oracle_lib):
    wl = synth.make_workload(n_int=12, n_ext=10, n_det=3, n_modes=4, n_bins=96, snr=12.0,
                             seed=11, ln_w="random")
    return wl, oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)


def test_routes_agree(small_noisy):
    wl, P = small_noisy
    for i in range(12):
        for e in range(0, 10, 3):
            d1, h1 = P.direct_phases(i, e)
            z, H = P.mode_components(i, e)
            d2, h2 = P.rotate_phases(z, H)
            scale = max(1.0, np.max(np.abs(d1)), np.max(np.abs(h1)))
            np.testing.assert_allclose(d1, d2, atol=1e-12 * scale)
            np.testing.assert_allclose(h1, h2, atol=1e-12 * scale)
            assert np.all(h1 >= 0.0)
            # H is Hermitian and positive semi-definite
            np.testing.assert_allclose(H, H.conj().T, atol=1e-15 * scale)
            assert np.min(np.linalg.eigvalsh(H)) > -1e-14 * scale


def test_residual_identity(small_noisy):
    # ln L = Re<d|h> - <h|h>/2 = <d|d>/2 - <d-h|d-h>/2, the right side built
    # from the generator's strain model and plain norms
    wl, P = small_noisy
    b, x, ev = wl.bank, wl.ext, wl.event
    wgt = 4.0 * b.w[None, :] / ev.psd
    dd = float(np.sum(wgt * np.abs(ev.data) ** 2))
    for (i, e, o) in [(0, 0, 0), (3, 7, 5), (11, 9, 31), (6, 2, 17)]:
        phi = 2 * np.pi * o / ev.n_phi
        hk = synth.signal_at_detectors(b.h[i], x.R[e], x.t[e], b.f, b.mode_m, phi, 1.0)
        res = float(np.sum(wgt * np.abs(ev.data - hk) ** 2))
        dh, hh = P.direct_phases(i, e)
        assert dh[o] - 0.5 * hh[o] == pytest.approx(0.5 * dd - 0.5 * res, abs=1e-10 * dd)
        assert dh[o] - 0.5 * hh[o] <= 0.5 * dd + 1e-12


@pytest.mark.parametrize("o_inj", [0, 5])
def test_noiseless_peak_at_injection(oracle_lib, o_inj):
    n_phi = 32
    wl = synth.make_workload(n_int=40, n_ext=24, n_det=3, n_modes=4, n_bins=128, snr=15.0,
                             seed=5, noise=False, insert_injection=True,
                             phi_inj=2 * np.pi * o_inj / n_phi)
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    ml = P.direct_grid_ml()
    i_star = wl.event.injection["i"]
    assert np.unravel_index(np.argmax(ml), ml.shape) == (i_star, 0)
    assert ml[i_star, 0] == pytest.approx(15.0 ** 2 / 2, abs=1e-9)
    dh, hh = P.direct_phases(i_star, 0)
    ll = [oracle_lib.lnl_ml(a, b) for a, b in zip(dh, hh)]
    assert int(np.argmax(ll)) == o_inj
    g, _ = P.eval_grid(0.0)
    ev = P.evidence(g)
    assert ev["arg"] == (i_star, 0, o_inj)
    assert ev["max_lnl_ml"] == pytest.approx(112.5, abs=1e-9)


def test_phase_marginal_matches_bessel_i0(oracle_lib):
    # single mode m = 2, fine phase grid: (1/N) sum_o exp(dh_o) -> I0(|z|);
    # rectangle-rule error ~ I_{N/2}(|z|)/I_0(|z|), negligible at N = 256
    wl = synth.make_workload(n_int=3, n_ext=3, n_det=2, n_modes=1, n_bins=64, snr=8.0, seed=3,
                             n_phi=256)
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    for i, e in [(0, 0), (1, 2), (2, 1)]:
        dh, hh = P.direct_phases(i, e)
        # single mode: dh_o = |z| cos(2 phi_o + a); period pi, hh constant
        np.testing.assert_allclose(dh[:128], dh[128:], atol=1e-12 * np.max(np.abs(dh)))
        np.testing.assert_allclose(hh, hh[0], rtol=1e-12)
        amp = math.sqrt(2.0 * np.mean(dh ** 2))
        lhs = np.log(np.mean(np.exp(dh - amp))) + amp
        rhs = math.log(special.i0e(amp)) + amp
        assert lhs == pytest.approx(rhs, abs=1e-12)


def test_noise_statistics_over_seeds(oracle_lib):
    # at the exact injection point, ln L^ML = (rho + n)^2 / 2 with n ~ N(0, 1):
    # mean rho^2/2 + 1/2, variance rho^2 + 1/2
    rho, vals = 6.0, []
    for seed in range(300):
        wl = synth.make_workload(n_int=2, n_ext=1, n_det=2, n_modes=2, n_bins=64, snr=rho,
                                 seed=1000 + seed, insert_injection=True)
        P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
        dh, hh = P.direct_phases(wl.event.injection["i"], 0)
        vals.append(dh[0] ** 2 / (2 * hh[0]))
    vals = np.array(vals)
    mean_sd = math.sqrt((rho ** 2 + 0.5) / len(vals))
    assert abs(vals.mean() - (rho ** 2 / 2 + 0.5)) < 5 * mean_sd
    assert 0.7 < vals.var(ddof=1) / (rho ** 2 + 0.5) < 1.35


# ---------------------------------------------------------------------------
# Eq. Z_sum and the effective sample sizes
# ---------------------------------------------------------------------------
def _brute_evidence(P, wl, n_phi):
    I, E = P.shape[:2]
    p = np.zeros((I, E, n_phi))
    ml = np.zeros((I, E, n_phi))
    for i in range(I):
        for e in range(E):
            dh, hh = P.direct_phases(i, e)
            for o in range(n_phi):
                lbar = math.exp(__import__("oracle").dist_marg(dh[o], hh[o], wl.event.u_min))
                p[i, e, o] = math.exp(wl.bank.ln_w[i] + wl.ext.ln_w[e]) * lbar
                ml[i, e, o] = __import__("oracle").lnl_ml(dh[o], hh[o])
    return p, ml


def test_evidence_brute_force(oracle_lib):
    wl = synth.make_workload(n_int=3, n_ext=4, n_det=2, n_modes=3, n_bins=48, snr=6.0, seed=7,
                             n_phi=4, ln_w="random")
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    p, ml = _brute_evidence(P, wl, 4)
    g, _ = P.eval_grid(0.0)
    ev = P.evidence(g)
    tot = p.sum()
    assert ev["ln_z"] == pytest.approx(math.log(tot / p.size), abs=1e-11)
    assert ev["n_eff"] == pytest.approx(tot ** 2 / np.sum(p ** 2), rel=1e-11)
    assert ev["n_eff_int"] == pytest.approx(tot ** 2 / np.sum(p.sum(axis=(1, 2)) ** 2), rel=1e-11)
    assert ev["n_eff_ext"] == pytest.approx(tot ** 2 / np.sum(p.sum(axis=(0, 2)) ** 2), rel=1e-11)
    np.testing.assert_allclose(ev["ln_p_int"], np.log(p.sum(axis=(1, 2))), atol=1e-11)
    np.testing.assert_allclose(ev["ln_p_ext"], np.log(p.sum(axis=(0, 2))), atol=1e-11)
    assert 1.0 <= ev["n_eff"] <= p.size
    # ML cut (Eq. coherent_ML_selection): keep phases within delta of the global max
    for delta in (1e-9, 0.5, 2.0, 1e6):
        g2, thr = P.eval_grid(delta)
        assert thr == pytest.approx(ml.max() - delta, abs=1e-9)
        keep = ml >= ml.max() - delta
        ev2 = P.evidence(g2)
        assert ev2["ln_z"] == pytest.approx(math.log(np.sum(p * keep) / p.size), abs=1e-11)
        assert ev2["n_marginalised"] == int(keep.sum())


def test_evidence_trivial_and_weight_shift(oracle_lib):
    wl = synth.make_workload(n_int=1, n_ext=1, n_det=2, n_modes=2, n_bins=64, snr=9.0, seed=4,
                             n_phi=1)
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    g, _ = P.eval_grid(0.0)
    dh, hh = P.direct_phases(0, 0)
    assert P.evidence(g)["ln_z"] == pytest.approx(
        oracle_lib.dist_marg(dh[0], hh[0], wl.event.u_min), abs=1e-12)
    wl = synth.make_workload(n_int=5, n_ext=6, n_det=2, n_modes=3, n_bins=64, snr=9.0, seed=4,
                             ln_w="random")
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    g, _ = P.eval_grid(0.0)
    ev = P.evidence(g)
    wl.bank.ln_w = wl.bank.ln_w + 1.75
    P2 = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    ev2 = P2.evidence(g)
    assert ev2["ln_z"] == pytest.approx(ev["ln_z"] + 1.75, abs=1e-12)
    assert ev2["n_eff"] == pytest.approx(ev["n_eff"], rel=1e-12)


def test_zero_data_gives_nonpositive_ln_z(oracle_lib):
    # d = 0: Re<d|h> = 0, so every Lbar <= 1 and ln Z <= 0
    wl = synth.make_workload(n_int=4, n_ext=5, n_det=2, n_modes=3, n_bins=64, snr=9.0, seed=8)
    wl.event.data = np.zeros_like(wl.event.data)
    P = oracle_lib.OracleProblem(wl.bank, wl.ext, wl.event)
    g, _ = P.eval_grid(0.0)
    assert P.evidence(g)["ln_z"] <= 0.0
    assert np.all(g["lnl_marg"] <= 0.0)
