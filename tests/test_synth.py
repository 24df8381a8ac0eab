"""Checks of the seeded input generator (geometry, harmonics, noise)."""
import math

import numpy as np
import pytest
from scipy import integrate

import synth


@pytest.mark.parametrize("l,m", [(2, 2), (2, -2), (2, 1), (2, -1), (3, 3), (3, -3), (4, 4), (4, -4)])
def test_spin_weighted_harmonics_normalised(l, m):
    # int |_{-2}Y_lm|^2 dOmega = 1 (the azimuthal factor has unit modulus)
    val, _ = integrate.quad(lambda th: synth.sYlm_m2(l, m, th) ** 2 * math.sin(th), 0, math.pi,
                            epsabs=1e-13)
    assert 2 * math.pi * val == pytest.approx(1.0, abs=1e-10)


def test_antenna_pattern_invariants():
    rng = np.random.default_rng(0)
    n = 200
    lat = np.arcsin(rng.uniform(-1, 1, n))
    lon = rng.uniform(0, 2 * np.pi, n)
    psi = rng.uniform(0, np.pi, n)
    for name in synth.DET_ORDER:
        _, D = synth.detector_geometry(name)
        fp, fc = synth.antenna_patterns(D, lat, lon, psi)
        fp2, fc2 = synth.antenna_patterns(D, lat, lon, psi + 0.37)
        # F+^2 + Fx^2 does not depend on psi
        np.testing.assert_allclose(fp ** 2 + fc ** 2, fp2 ** 2 + fc2 ** 2, atol=1e-12)
        # psi -> psi + pi/2 flips the sign of both
        fp3, fc3 = synth.antenna_patterns(D, lat, lon, psi + np.pi / 2)
        np.testing.assert_allclose(fp3, -fp, atol=1e-12)
        np.testing.assert_allclose(fc3, -fc, atol=1e-12)
        assert np.all(fp ** 2 + fc ** 2 <= 1.0 + 1e-12)


def test_arrival_time_delays_bounded():
    wl = synth.make_workload(n_int=2, n_ext=500, n_det=3, n_modes=4, n_bins=32, seed=1)
    dt = wl.ext.t - wl.ext.t_geo[:, None]
    assert np.max(np.abs(dt)) <= synth.R_EARTH / synth.C_LIGHT + 1e-12


def test_quadrature_weights_integrate_linear_exactly():
    f, w = synth.freq_grid(257)
    assert np.sum(w) == pytest.approx(1024 - 20, rel=1e-13)
    assert np.sum(w * f) == pytest.approx(0.5 * (1024 ** 2 - 20 ** 2), rel=1e-13)


def test_noise_normalisation():
    # Re<n|h> ~ N(0, <h|h>) under the discrete inner product
    f, w = synth.freq_grid(64)
    psd = synth.analytic_psd(f)
    rng = np.random.default_rng(3)
    h = (1 + 0.5j) * f ** (-7 / 6)
    hh = np.sum(4 * w * np.abs(h) ** 2 / psd)
    sig = np.sqrt(psd / (4 * w))
    n = sig * (rng.standard_normal((20000, 64)) + 1j * rng.standard_normal((20000, 64)))
    x = np.sum(4 * w * (n * np.conj(h)).real / psd, axis=1)
    assert x.var() / hh == pytest.approx(1.0, abs=0.05)


def test_seeded_reproducible():
    a = synth.make_workload(n_int=8, n_ext=4, n_det=2, n_modes=3, n_bins=16, seed=9)
    b = synth.make_workload(n_int=8, n_ext=4, n_det=2, n_modes=3, n_bins=16, seed=9)
    assert np.array_equal(a.bank.h, b.bank.h) and np.array_equal(a.event.data, b.event.data)
    assert np.array_equal(a.ext.R, b.ext.R)
