"""Pins of the oracle's relative-binning weights (App. A, Eqs. dh_weights,
hh_weights, d_h, h_h) against fine-grid inner products computed directly.

Relative binning is exact whenever the ratio of a waveform to the reference
is linear between adjacent nodes (the hat functions interpolate it exactly),
in particular for the reference itself (the hat functions sum to one).  The
pins build such waveforms on the fine grid and compare the binned sums with
plain fine-grid sums; a last check bounds the approximation for bank rows
near the reference at the time shifts of the workload's extrinsic samples.
"""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def rbw():
    import oracle
    oracle.build()
    rw = synth.make_rb_workload(n_int=24, n_ext=8, n_det=2, n_modes=3, n_bins=120, n_fine=12000, seed=11)
    w = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    return oracle, rw, w


def fine_ip(rw, d, a, b):
    """<a|b>_d = sum_n 4 dff a b^* / S_d on the fine grid."""
    return np.sum(4.0 * rw.dff * a * np.conj(b) / rw.psd_fine[d])


def shift(rw, d):
    return np.exp(-2j * np.pi * rw.f_fine * rw.t0[d])


def test_reference_is_exact(rbw):
    """h = h0 (arriving at t0): sum_b W^{<d|h>} h0^*(f_b) = <d|h0> and
    sum_b W^{<h|h>} h0 h0'^*(f_b) = <h0|h0'> on the fine grid."""
    oracle, rw, (wdh, whh) = rbw
    D, M = rw.psd_fine.shape[0], rw.h0_fine.shape[0]
    for d in range(D):
        h0d = rw.h0_fine * shift(rw, d)[None, :]
        at = h0d[:, rw.nodes]
        for m in range(M):
            got = np.sum(wdh[d, m] * np.conj(at[m]))
            assert got == pytest.approx(fine_ip(rw, d, rw.data_fine[d], h0d[m]), rel=1e-11)
            for mp in range(M):
                got = np.sum(whh[d, m, mp] * at[m] * np.conj(at[mp]))
                assert got == pytest.approx(fine_ip(rw, d, h0d[m], h0d[mp]), rel=1e-11)


def test_exact_for_piecewise_linear_ratio(rbw):
    """h_m = h0_m r_m with r_m linear between nodes (random complex node values)."""
    oracle, rw, (wdh, whh) = rbw
    rng = np.random.default_rng(5)
    D, M = rw.psd_fine.shape[0], rw.h0_fine.shape[0]
    fb = rw.f_fine[rw.nodes]
    for d in range(D):
        h0d = rw.h0_fine * shift(rw, d)[None, :]
        for m in range(M):
            rb = rng.standard_normal(len(fb)) + 1j * rng.standard_normal(len(fb))
            r = np.interp(rw.f_fine, fb, rb.real) + 1j * np.interp(rw.f_fine, fb, rb.imag)
            h = h0d[m] * r
            got = np.sum(wdh[d, m] * np.conj(h[rw.nodes]))
            assert got == pytest.approx(fine_ip(rw, d, rw.data_fine[d], h), rel=1e-10)
            # <h_m | h0_m'>: the product's ratio r_m * 1 is linear too
            for mp in range(M):
                got = np.sum(whh[d, m, mp] * h[rw.nodes] * np.conj(h0d[mp, rw.nodes]))
                assert got == pytest.approx(fine_ip(rw, d, h, h0d[mp]), rel=1e-10)


def test_weights_structure(rbw):
    """W^{<h|h>} is Hermitian in the mode pair, its diagonal real and positive."""
    oracle, rw, (wdh, whh) = rbw
    np.testing.assert_allclose(whh, np.conj(np.swapaxes(whh, 1, 2)), rtol=1e-12, atol=0)
    diag = np.einsum("dmmb->dmb", whh)
    assert np.all(diag.real > 0)
    np.testing.assert_allclose(diag.imag, 0.0, atol=1e-12 * np.abs(diag).max())


def test_pipeline_route_o2_uses_the_weights(rbw):
    """The oracle's per-mode components with relative binning equal the
    fine-grid sums for the reference row at the reference's arrival times
    (exact), and approximate them for nearby rows at the samples' time shifts
    (an accuracy check of the approximation, not a pin: 4e-4 relative with 120
    nodes here, inside the paper's "better than 1%")."""
    oracle, rw, (wdh, whh) = rbw
    import copy
    ext0 = copy.deepcopy(rw.ext)
    ext0.t[:] = rw.t0[None, :]
    for ext, rows, tol_z, tol_h in ((ext0, (0,), 1e-10, 1e-10), (rw.ext, (0, 3, 9, 20), 2e-3, 1e-5)):
        P = oracle.OracleProblem(rw.bank, ext, rw.event, rb=(wdh, whh))
        for i in rows:
            hf = rw.rows_fine(i)[0]
            for e in (0, 5):
                z, H = P.mode_components(i, e)
                zt = np.zeros_like(z)
                Ht = np.zeros_like(H)
                for d in range(rw.psd_fine.shape[0]):
                    sh = np.exp(-2j * np.pi * rw.f_fine * ext.t[e, d])
                    for m in range(len(z)):
                        zt[m] += ext.R[e, d, m] * np.conj(fine_ip(rw, d, rw.data_fine[d], hf[m] * sh))
                        for mp in range(len(z)):
                            Ht[m, mp] += ext.R[e, d, m] * np.conj(ext.R[e, d, mp]) * fine_ip(rw, d, hf[m], hf[mp])
                assert np.max(np.abs(z - zt)) <= tol_z * np.max(np.abs(zt)), (i, e)
                assert np.max(np.abs(H - Ht)) <= tol_h * np.max(np.abs(Ht)), (i, e)


def test_preselection_uses_the_weights(rbw):
    """Pre-selection with relative binning on the reference row, on a time grid
    at the reference's arrival times: the fine-grid projection of App. B."""
    oracle, rw, (wdh, whh) = rbw
    D, M = rw.psd_fine.shape[0], rw.h0_fine.shape[0]
    pol = synth.row_polarisation_factors(rw.bank, np.full(rw.bank.h.shape[0], 0.3))
    t_grid = rw.t0[:, None].copy()
    P = oracle.PreselProblem(rw.bank.f, rw.bank.w, rw.bank.mode_m, rw.bank.h, pol, rw.event.psd,
                             rw.event.data, t_grid, n_phi=4, rb=(wdh, whh))
    for k in range(D):
        g = P.grid(0, k)
        om = np.sqrt(4.0 * rw.dff / rw.psd_fine[k])
        vd = np.concatenate([rw.data_fine[k].real * om, rw.data_fine[k].imag * om])
        for o in range(4):
            cols = []
            for p in range(2):
                tpl = sum(pol[0, m, p] * rw.h0_fine[m] * np.exp(1j * rw.bank.mode_m[m] * 2 * np.pi * o / 4)
                          for m in range(M)) * shift(rw, k)
                cols.append(np.concatenate([tpl.real * om, tpl.imag * om]))
            A = np.stack(cols, axis=1)
            x, *_ = np.linalg.lstsq(A, vd, rcond=None)
            res = vd - A @ x
            assert g[o, 0] == pytest.approx(0.5 * (vd @ vd - res @ res), rel=1e-9)


# --------------------------------------------------------------------------
# polarisation-resolved (precessing) bank: weights per (mode, polarisation)
# component, W_{kmpb} and W_{kmm'pp'b} (Eqs. dh_weights, hh_weights)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def rbp():
    import oracle
    oracle.build()
    rw = synth.make_rb_workload(n_int=12, n_ext=6, n_det=2, n_modes=3, n_bins=120, n_fine=12000, seed=13,
                                precessing=True)
    w = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    return oracle, rw, w


def test_polarisation_resolved_reference_is_exact(rbp):
    """Every component j = (m, p) of a precessing reference: the binned sums
    equal the fine-grid <d|h0_j> and <h0_j|h0_j'>."""
    oracle, rw, (wdh, whh) = rbp
    D, J = rw.psd_fine.shape[0], rw.h0_fine.shape[0]
    assert wdh.shape == (D, J, len(rw.nodes)) and whh.shape == (D, J, J, len(rw.nodes))
    for d in range(D):
        h0d = rw.h0_fine * shift(rw, d)[None, :]
        at = h0d[:, rw.nodes]
        for j in range(J):
            assert np.sum(wdh[d, j] * np.conj(at[j])) == pytest.approx(
                fine_ip(rw, d, rw.data_fine[d], h0d[j]), rel=1e-11)
            for jp in range(J):
                assert np.sum(whh[d, j, jp] * at[j] * np.conj(at[jp])) == pytest.approx(
                    fine_ip(rw, d, h0d[j], h0d[jp]), rel=1e-11)


def test_polarisation_resolved_pipeline(rbp):
    """Route O2 of a precessing bank with the component weights: per-mode
    components z_m = sum_{d,p} F_edp conj<d|h_mp T> and overlaps H_mm' =
    sum_{d,p,p'} F_edp F_edp' <h_mp|h_m'p'> equal the fine-grid sums for the
    reference row at the reference's arrival times."""
    oracle, rw, (wdh, whh) = rbp
    import copy
    ext0 = copy.deepcopy(rw.ext)
    ext0.t[:] = rw.t0[None, :]
    P = oracle.OracleProblem(rw.bank, ext0, rw.event, rb=(wdh, whh))
    hf = rw.rows_fine(0)[0]  # [M, 2, N]
    M = hf.shape[0]
    for e in (0, 3):
        z, H = P.mode_components(0, e)
        zt = np.zeros(M, np.complex128)
        Ht = np.zeros((M, M), np.complex128)
        for d in range(rw.psd_fine.shape[0]):
            sh = shift(rw, d)
            F = ext0.F[e, d]
            for m in range(M):
                for p in range(2):
                    zt[m] += F[p] * np.conj(fine_ip(rw, d, rw.data_fine[d], hf[m, p] * sh))
                    for mp in range(M):
                        for pp in range(2):
                            Ht[m, mp] += F[p] * F[pp] * fine_ip(rw, d, hf[m, p], hf[mp, pp])
        assert np.max(np.abs(z - zt)) <= 1e-10 * np.max(np.abs(zt))
        assert np.max(np.abs(H - Ht)) <= 1e-10 * np.max(np.abs(Ht))


def test_polarisation_resolved_preselection_uses_the_component_weights(rbp):
    """Pre-selection of a precessing bank with the component weights, on the
    reference row at the reference's arrival times: the fine-grid projection of
    App. B onto the two real templates sum_m h_mp e^{i m phi_o} T_k, p = +, x."""
    oracle, rw, (wdh, whh) = rbp
    D = rw.psd_fine.shape[0]
    hf = rw.rows_fine(0)[0]  # [M, 2, N]
    M = hf.shape[0]
    P = oracle.PreselProblem(rw.bank.f, rw.bank.w, rw.bank.mode_m, rw.bank.h, None, rw.event.psd,
                             rw.event.data, rw.t0[:, None].copy(), n_phi=4, rb=(wdh, whh))
    for k in range(D):
        g = P.grid(0, k)
        om = np.sqrt(4.0 * rw.dff / rw.psd_fine[k])
        vd = np.concatenate([rw.data_fine[k].real * om, rw.data_fine[k].imag * om])
        for o in range(4):
            cols = []
            for p in range(2):
                tpl = sum(hf[m, p] * np.exp(1j * rw.bank.mode_m[m] * 2 * np.pi * o / 4) for m in range(M)) \
                    * shift(rw, k)
                cols.append(np.concatenate([tpl.real * om, tpl.imag * om]))
            A = np.stack(cols, axis=1)
            x, *_ = np.linalg.lstsq(A, vd, rcond=None)
            res = vd - A @ x
            assert g[o, 0] == pytest.approx(0.5 * (vd @ vd - res @ res), rel=1e-9)


def test_fixed_inclination_components_reduce_to_mode_weights():
    """A reference whose polarisations are h0_mp = K_mp h0_m with constant K:
    the factor cancels in both ratios, so W_{k(m,p)b} = W_{kmb} and
    W_{k(m,p)(m',p')b} = W_{kmm'b}; with those weights a fixed-inclination
    polarisation-resolved bank gives the mode bank's likelihood with
    R_edm = F_ed+ K_m+ + F_edx K_mx, pair by pair."""
    import copy
    import oracle
    oracle.build()
    rw = synth.make_rb_workload(n_int=10, n_ext=7, n_det=2, n_modes=3, n_bins=100, n_fine=10000, seed=17)
    iota = np.arccos(0.35)
    K = np.array([synth.polarisation_factors(int(l), int(m), iota)
                  for l, m in zip(rw.bank.mode_l, rw.bank.mode_m)])  # [M, 2]
    M = K.shape[0]
    h0p = (rw.h0_fine[:, None, :] * K[:, :, None]).reshape(2 * M, -1)
    wdh, whh = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    pdh, phh = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, h0p, rw.nodes, rw.t0)
    D, B = wdh.shape[0], wdh.shape[-1]
    np.testing.assert_allclose(pdh.reshape(D, M, 2, B), np.repeat(wdh[:, :, None, :], 2, axis=2), rtol=1e-11,
                               atol=1e-13 * np.abs(wdh).max())
    np.testing.assert_allclose(phh.reshape(D, M, 2, M, 2, B),
                               np.broadcast_to(whh[:, :, None, :, None, :], (D, M, 2, M, 2, B)), rtol=1e-11,
                               atol=1e-13 * np.abs(whh).max())
    bank_p = synth.Bank(**{**rw.bank.__dict__, "h": rw.bank.h[:, :, None, :] * K[None, :, :, None]})
    ext_k = copy.deepcopy(rw.ext)
    ext_k.R = np.einsum("edp,mp->edm", rw.ext.F, K)
    Pp = oracle.OracleProblem(bank_p, rw.ext, rw.event, rb=(pdh, phh))
    Pn = oracle.OracleProblem(rw.bank, ext_k, rw.event, rb=(wdh, whh))
    pi, pe = np.divmod(np.arange(10 * 7), 7)
    a, b = Pp.eval_pairs(pi, pe), Pn.eval_pairs(pi, pe)
    np.testing.assert_allclose(a["lnl_marg"], b["lnl_marg"], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(a["lnl_ml_max"], b["lnl_ml_max"], rtol=1e-10, atol=1e-10)
