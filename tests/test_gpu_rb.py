"""Relative binning (App. A) on the device, through the C ABI, against the FP64
oracle with the same weights.

* dotpe_rb_weights (FP64 on the device) equals the oracle's weights to FP64
  rounding (|dW| <= 1e-11 max|W|).
* An event evaluated with the weights (per-mode data weights, complex
  mode-pair <h|h> weights) meets the coherent path's tolerances against the
  oracle's route O2 with the same weights, all pairs: 1e-3 per pair for FP32
  and split fp16 (whose hi*hi products accumulate in three interleaved TMEM
  sets; the peak here is ln L^ML ~ 230); |d ln Z| <= 1e-2.
* The pre-selection with the weights (one time-grid operand per mode) meets
  its split tolerance 2e-3 + 1e-4 ln L^ML against the oracle.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-3  # per pair, split precision


@pytest.fixture(scope="module")
def dpx():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    ctx = dp.dotpe_create(0)
    yield dp, ctx
    dp.dotpe_destroy(ctx)


@pytest.fixture(scope="module")
def rbw():
    import oracle
    # 1,000 rows (a ragged row tile), 200 samples, the paper's N_f = 378 nodes on a 65,536-point grid
    rw = synth.make_rb_workload(n_int=1000, n_ext=200, n_det=3, n_modes=4, n_bins=378, n_fine=65536, seed=51,
                                snr=20.0)
    w = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    return rw, w


def test_weights_kernel_matches_oracle(dpx, rbw):
    dp, ctx = dpx
    rw, (wdh, whh) = rbw
    gdh, ghh = dp.dotpe_rb_weights(ctx, rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    assert np.max(np.abs(gdh - wdh)) <= 1e-11 * np.max(np.abs(wdh))
    assert np.max(np.abs(ghh - whh)) <= 1e-11 * np.max(np.abs(whh))


def test_weights_errors(dpx, rbw):
    dp, ctx = dpx
    rw, _ = rbw
    bad = rw.nodes.copy()
    bad[5] = bad[4]
    with pytest.raises(dp.DotpeError) as ei:
        dp.dotpe_rb_weights(ctx, rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, bad, rw.t0)
    assert ei.value.status == dp.DOTPE_E_INVALID
    h0 = rw.h0_fine.copy()
    h0[1, rw.nodes[7]] = 0.0
    with pytest.raises(dp.DotpeError) as ei:
        dp.dotpe_rb_weights(ctx, rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, h0, rw.nodes, rw.t0)
    assert ei.value.status == dp.DOTPE_E_INVALID and "vanishes" in str(ei.value)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "mixed"])
def test_event_with_weights_against_oracle(dpx, rbw, precision):
    dp, ctx = dpx
    rw, (wdh, whh) = rbw
    import oracle
    P = oracle.OracleProblem(rw.bank, rw.ext, rw.event, rb=(wdh, whh))
    grid, _ = P.eval_grid(0.0)
    ref = P.evidence(grid)
    bank = rw.bank
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        I, E = bank.h.shape[0], rw.ext.t.shape[0]
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, None, None, rw.ext.t, rw.ext.R, rw.ext.ln_w,
                                    n_phi=rw.event.n_phi, u_min=rw.event.u_min, cut_delta=0.0,
                                    precision=precision, flags=dp.DOTPE_FLAG_STORE_LNL, rb=(wdh, whh))
        dp.dotpe_event_wait(ctx, eid, 120.0)
        ev = dp.dotpe_evidence(ctx, eid)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E)
        ml = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E, what=dp.DOTPE_LNL_ML_MAX)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    d1 = np.abs(lnl - grid["lnl_marg"])
    d2 = np.abs(ml - grid["lnl_ml_max"])
    ml_ref = grid["lnl_ml_max"]
    if precision == "mixed":
        # pairs within 30 of the maximum are refined (split bound); the others keep
        # the single-pass fp16 bound, with the binned data's Cauchy-Schwarz scale
        # max_m sum |W^{<d|h>}|^2 / W^{<h|h>}_{mm} in place of <d|d>
        near = ml_ref >= ml_ref.max() - 30.0
        u = 2.0 ** -11
        dd = max(float(np.sum(np.abs(wdh[:, m]) ** 2 / whh[:, m, m].real)) for m in range(wdh.shape[1]))
        mlp = np.maximum(ml_ref, 0)
        far_tol = 2e-2 + 4 * u * mlp + 2 * u * np.sqrt(2 * mlp + 1) * np.sqrt(dd)
        tol = np.where(near, SPLIT_TOL, far_tol)
    elif precision == "fp16x3":
        tol = np.full_like(ml_ref, SPLIT_TOL)
    else:
        tol = np.full_like(ml_ref, 1e-3)
    print(f"rb event {precision}: max |d ln Lbar| {d1.max():.3e}, max |d ln L^ML| {d2.max():.3e}, "
          f"d ln Z {ev['ln_z'] - ref['ln_z']:.3e}, peak ln L^ML {ml_ref.max():.1f}")
    assert np.all(d1 <= tol)
    assert np.all(d2 <= tol)
    assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2
    assert (ev["arg_i"], ev["arg_e"]) == ref["arg"][:2]


def test_preselection_with_weights_against_oracle(dpx, rbw):
    dp, ctx = dpx
    rw, (wdh, whh) = rbw
    import oracle
    I = rw.bank.h.shape[0]
    cos_iota = np.random.default_rng(52).uniform(-1, 1, I)
    cos_iota[0] = rw.event.injection["cos_iota"]
    pol = synth.row_polarisation_factors(rw.bank, cos_iota)
    D = rw.psd_fine.shape[0]
    t_grid = rw.t0[:, None] + (np.arange(48) - 24)[None, :] * 2.5e-4
    Pq = oracle.PreselProblem(rw.bank.f, rw.bank.w, rw.bank.mode_m, rw.bank.h, pol, rw.event.psd, rw.event.data,
                              t_grid, n_phi=32, rb=(wdh, whh))
    ref = Pq.run(delta=20.0)
    bank = rw.bank
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w, pol=pol)
    try:
        out = {}
        for precision in ("fp16x3", "bf16x3"):
            out[precision] = dp.dotpe_preselect(ctx, bid, 0, I, None, None, t_grid, n_phi=32, delta=20.0,
                                                precision=precision, rb=(wdh, whh))
    finally:
        dp.dotpe_bank_release(ctx, bid)
    tol = 2e-3 + 1e-4 * np.abs(ref["ml"])
    for precision, r in out.items():
        d = np.abs(r["lnl_ml"] - ref["ml"])
        print(f"rb presel {precision}: max |d ln L^ML_ik| {d.max():.3e} (up to {ref['ml'].max():.1f})")
        assert np.all(d <= tol), (precision, float(d.max()))
        # the kernel's maximum row is the oracle's, or ties it within the tolerance
        assert abs(ref["lnl_inco"][r["arg_i"]] - ref["lnl_inco"].max()) <= tol.sum(1).max()
        # the injected (reference) row is kept
        assert 0 in set(r["selected"].tolist())


# --------------------------------------------------------------------------
# polarisation-resolved (precessing) bank: weights per (mode, polarisation)
# component, W_{kmpb} and W_{kmm'pp'b} (App. A as written)
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def rbp():
    import oracle
    # 8 components (4 modes x 2 polarisations), 378 nodes, a ragged row tile
    rw = synth.make_rb_workload(n_int=520, n_ext=150, n_det=3, n_modes=4, n_bins=378, n_fine=65536, seed=57,
                                snr=20.0, precessing=True)
    w = oracle.rb_weights(rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    return rw, w


def test_component_weights_kernel_matches_oracle(dpx, rbp):
    dp, ctx = dpx
    rw, (wdh, whh) = rbp
    gdh, ghh = dp.dotpe_rb_weights(ctx, rw.f_fine, rw.dff, rw.psd_fine, rw.data_fine, rw.h0_fine, rw.nodes, rw.t0)
    assert gdh.shape == (3, 8, 378) and ghh.shape == (3, 8, 8, 378)
    assert np.max(np.abs(gdh - wdh)) <= 1e-11 * np.max(np.abs(wdh))
    assert np.max(np.abs(ghh - whh)) <= 1e-11 * np.max(np.abs(whh))


def test_precessing_preselection_with_component_weights(dpx, rbp):
    """Pre-selection of the 520-row precessing bank with the component weights
    (one FP32 time-grid operand per (mode, polarisation) component, 150 times:
    two passes of the kernel's 128 time slots) against the oracle with the same
    weights: the split bound 2e-3 + 1e-4 ln L^ML per (row, detector), the
    incoherent sums within the detectors' bounds, the kept set away from the
    threshold, the (o, t) within the bound; a slice (its own records) equals
    the whole-bank call (the cached records) bit for bit."""
    dp, ctx = dpx
    rw, (wdh, whh) = rbp
    import oracle
    I, D = rw.bank.h.shape[0], rw.psd_fine.shape[0]
    t_grid = rw.t0[:, None] + (np.arange(150) - 75)[None, :] * 2.5e-4
    P = oracle.PreselProblem(rw.bank.f, rw.bank.w, rw.bank.mode_m, rw.bank.h, None, rw.event.psd, rw.event.data,
                             t_grid, n_phi=32, rb=(wdh, whh))
    ref = P.run(delta=20.0)
    bid = dp.dotpe_bank_load(ctx, rw.bank.h, rw.bank.f, rw.bank.w, rw.bank.mode_m, rw.bank.ln_w)
    try:
        part = dp.dotpe_preselect(ctx, bid, 100, 200, None, None, t_grid, n_phi=32, delta=20.0, precision="fp32",
                                  rb=(wdh, whh))
        r = dp.dotpe_preselect(ctx, bid, 0, I, None, None, t_grid, n_phi=32, delta=20.0, precision="fp32",
                               rb=(wdh, whh))
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_preselect(ctx, bid, 0, I, None, None, t_grid, n_phi=32, delta=20.0, precision="bf16x3",
                               rb=(wdh, whh))
        assert ei.value.status == dp.DOTPE_E_UNSUPPORTED
    finally:
        dp.dotpe_bank_release(ctx, bid)
    assert r["device_status"] == 0
    tol = 2e-3 + 1e-4 * np.abs(ref["ml"])
    d = np.abs(r["lnl_ml"] - ref["ml"])
    print(f"rb presel precessing fp32: max |d ln L^ML_ik| {d.max():.3e} (up to {ref['ml'].max():.1f})")
    assert np.all(d <= tol), float(d.max())
    tol_i = tol.sum(axis=1)
    assert np.all(np.abs(r["lnl_inco"] - ref["lnl_inco"]) <= tol_i)
    keep_gpu = np.zeros(I, bool)
    keep_gpu[r["selected"]] = True
    clear = np.abs(ref["lnl_inco"] - ref["threshold"]) > 2 * tol_i.max()
    np.testing.assert_array_equal(keep_gpu[clear], ref["keep"][clear])
    for i in (0, 259, I - 1, int(r["arg_i"])):
        for k in range(D):
            g = P.grid(i, k)
            o, t = r["arg_ot"][i, k]
            assert g[o, t] >= g.max() - 2 * tol[i, k]
    np.testing.assert_array_equal(part["lnl_ml"], r["lnl_ml"][100:200])
    np.testing.assert_array_equal(part["arg_ot"], r["arg_ot"][100:200])


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "mixed"])
def test_precessing_event_with_component_weights(dpx, rbp, precision):
    """A polarisation-resolved event with relative binning against the
    oracle's route O2 with the same component weights, all pairs: the
    coherent path's bounds (K = 4B here, Kpad = 1536): split precision 1e-3,
    FP32 with an ln L^ML-proportional term (the peak here is ln L^ML ~ 200)."""
    dp, ctx = dpx
    rw, (wdh, whh) = rbp
    import oracle
    P = oracle.OracleProblem(rw.bank, rw.ext, rw.event, rb=(wdh, whh))
    grid, _ = P.eval_grid(0.0)
    ref = P.evidence(grid)
    bank = rw.bank
    I, E = bank.h.shape[0], rw.ext.t.shape[0]
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, None, None, rw.ext.t, None, rw.ext.ln_w,
                                    n_phi=rw.event.n_phi, u_min=rw.event.u_min, cut_delta=0.0,
                                    precision=precision, flags=dp.DOTPE_FLAG_STORE_LNL, rb=(wdh, whh), F=rw.ext.F)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        ev = dp.dotpe_evidence(ctx, eid)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E)
        ml = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E, what=dp.DOTPE_LNL_ML_MAX)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    ml_ref = grid["lnl_ml_max"]
    mlp = np.maximum(ml_ref, 0)
    if precision == "mixed":
        near = ml_ref >= ml_ref.max() - 30.0
        u = 2.0 ** -11
        J = wdh.shape[1]
        dd = max(float(np.sum(np.abs(wdh[:, j]) ** 2 / whh[:, j, j].real)) for j in range(J))
        far_tol = 2e-2 + 4 * u * mlp + 2 * u * np.sqrt(2 * mlp + 1) * np.sqrt(dd)
        tol = np.where(near, SPLIT_TOL, far_tol)
    elif precision == "fp16x3":
        tol = np.full_like(mlp, SPLIT_TOL)
    else:
        # FP32 operands (weights, phases, records) carry ~2^-17 relative error,
        # which moves ln L^ML = z^2 / 2 hh by about twice that, relative
        tol = 1e-3 + 2.0 ** -16 * mlp
    d1 = np.abs(lnl - grid["lnl_marg"])
    d2 = np.abs(ml - ml_ref)
    print(f"precessing rb event {precision}: max |d ln Lbar| {d1.max():.3e}, max |d ln L^ML| {d2.max():.3e}, "
          f"d ln Z {ev['ln_z'] - ref['ln_z']:.3e}, peak ln L^ML {ml_ref.max():.1f}")
    assert np.all(d1 <= tol)
    assert np.all(d2 <= tol)
    assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2
    assert (ev["arg_i"], ev["arg_e"]) == ref["arg"][:2]
