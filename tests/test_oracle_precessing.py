"""Pins of the oracle for polarisation-resolved (precessing) banks (Sec. IV.A
general case: Eqs. dh_ieo, hh_ieo with the polarisation index p and real
antenna patterns F_{edp}).

* Route O2 (per-mode, per-polarisation components) equals route O1 (the
  detector strain built directly) on a small problem.
* A polarisation-resolved bank built from a non-precessing one at a fixed
  inclination, h_{imp} = K_{mp}(iota) h_{im}, gives exactly the non-precessing
  likelihood with R_{edm} = F_{ed+} K_{m+}(iota) + F_{edx} K_{mx}(iota).
* A noiseless injection peaks at its own (i, e, o) with ln L^ML = SNR^2 / 2.
"""
import copy

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def test_route_o2_equals_route_o1(orc):
    wl = synth.make_precessing_workload(4, 6, 3, 4, 24, seed=3, n_phi=8)
    P = orc.OracleProblem(wl.bank, wl.ext, wl.event)
    for i in range(4):
        for e in range(6):
            dh1, hh1 = P.direct_phases(i, e)
            z, H = P.mode_components(i, e)
            dh2, hh2 = P.rotate_phases(z, H)
            np.testing.assert_allclose(dh2, dh1, rtol=1e-12, atol=1e-12 * np.abs(dh1).max())
            np.testing.assert_allclose(hh2, hh1, rtol=1e-12)


def test_fixed_inclination_reduces_to_the_mode_response(orc):
    wl = synth.make_workload(n_int=5, n_ext=7, n_det=2, n_modes=4, n_bins=32, seed=4, n_phi=8)
    iota = np.arccos(0.4)
    M = wl.bank.mode_m.shape[0]
    K = np.array([synth.polarisation_factors(int(l), int(m), iota)
                  for l, m in zip(wl.bank.mode_l, wl.bank.mode_m)])  # [M, 2]
    hp = wl.bank.h[:, :, None, :] * K[None, :, :, None]               # [I, M, 2, B]
    bank_p = synth.Bank(**{**wl.bank.__dict__, "h": hp})
    ext_fixed = copy.deepcopy(wl.ext)
    ext_fixed.R = np.einsum("edp,mp->edm", wl.ext.F, K)
    Pp = orc.OracleProblem(bank_p, wl.ext, wl.event)
    Pn = orc.OracleProblem(wl.bank, ext_fixed, wl.event)
    pi, pe = np.divmod(np.arange(5 * 7), 7)
    a = Pp.eval_pairs(pi, pe)
    b = Pn.eval_pairs(pi, pe)
    np.testing.assert_allclose(a["lnl_marg"], b["lnl_marg"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a["lnl_ml_max"], b["lnl_ml_max"], rtol=1e-12, atol=1e-12)


def test_noiseless_injection_peaks_at_snr_squared_over_two(orc):
    wl = synth.make_precessing_workload(16, 6, 3, 4, 64, snr=12.0, seed=5, n_phi=8, noise=False,
                                        insert_injection=True)
    P = orc.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ev = P.evidence(grid)
    assert ev["max_lnl_ml"] == pytest.approx(0.5 * 12.0 ** 2, rel=1e-10)
    assert ev["arg"] == (wl.event.injection["i"], 0, 0)
