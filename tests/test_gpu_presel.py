"""Parity of the pre-selection kernel (Sec. IV.D, App. B) with the FP64 oracle,
through the C ABI.

Tolerances on ln L^ML_{ik} = max_{o,t} ln L^ML_{ikot} (and on ln L^inco.ML,
summed over detectors):
  fp16x3 / bf16x3 (split): |d| <= 2e-3 + 1e-4 ln L^ML.  The tensor cores add
    every MMA's products into one FP32 accumulator with truncation: Kpad/16
    steps per pass, three passes, i.e. up to ~3 (Kpad/16) 2^-24 relative in Z
    (~6e-6 at B = 256, ~1.1e-5 at B = 512), twice that in ln L^ML, then the
    FP32 epilogue (<h|h> from FP32 mode overlaps, the 2x2 pseudo-inverse,
    conditioned up to 1/rank_tol) adds a few 1e-6 relative.
  fp16 (single pass): the coherent kernel's single-pass bound with the
    detector's own <d_k|d_k>:  2e-2 + 4u ln L^ML + 2u sqrt(2 ln L^ML + 1)
    sqrt(<d_k|d_k>), u = 2^-11.
The selection must agree with the oracle's on every row whose oracle
ln L^inco.ML is farther from the oracle's threshold than the tolerance.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

U16 = 2.0 ** -11


def split_tol(ml):
    return 2e-3 + 1e-4 * np.abs(ml)


def fp16_tol(ml, dd_k):
    ml = np.maximum(ml, 0.0)
    return 2e-2 + 4 * U16 * ml + 2 * U16 * np.sqrt(2 * ml + 1) * np.sqrt(dd_k)


@pytest.fixture(scope="module")
def dpx():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    ctx = dp.dotpe_create(0)
    yield dp, ctx
    dp.dotpe_destroy(ctx)


def load_bank(dp, ctx, wl, ps):
    return dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w, pol=ps.pol)


def oracle_rows(wl, ps, rows, n_phi, delta=20.0):
    import oracle
    rows = np.asarray(rows, dtype=np.int64)
    P = oracle.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h[rows], ps.pol[rows],
                             wl.event.psd, wl.event.data, ps.t_grid, n_phi=n_phi)
    return P, P.run(delta=delta)


def dd_per_detector(wl):
    return np.sum(4.0 * wl.bank.w[None, :] * np.abs(wl.event.data) ** 2 / wl.event.psd, axis=1)


@pytest.fixture(scope="module")
def small():
    # 1,000 rows (a ragged last row tile), 40 time points (padded to 64 columns per detector)
    wl = synth.make_workload(n_int=1000, n_ext=4, n_det=3, n_modes=4, n_bins=256, seed=41, snr=15.0)
    ps = synth.make_presel_inputs(wl, n_t=40, dt=1.5e-3, seed=42)
    _, ref = oracle_rows(wl, ps, np.arange(1000), 32)
    return wl, ps, ref


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "fp16"])
def test_small_all_rows_against_oracle(dpx, small, precision):
    dp, ctx = dpx
    wl, ps, ref = small
    bid = load_bank(dp, ctx, wl, ps)
    try:
        r = dp.dotpe_preselect(ctx, bid, 0, 1000, wl.event.psd, wl.event.data, ps.t_grid, n_phi=32,
                               delta=20.0, precision=precision)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    assert r["device_status"] == 0
    ml_ref = ref["ml"]
    if precision == "fp16":
        tol = fp16_tol(ml_ref, dd_per_detector(wl)[None, :])
    else:
        tol = split_tol(ml_ref)
    d = np.abs(r["lnl_ml"] - ml_ref)
    print(f"presel {precision}: max |d ln L^ML_ik| {d.max():.3e} (ln L^ML up to {ml_ref.max():.1f})")
    assert np.all(d <= tol), (precision, float(d.max()))
    tol_i = tol.sum(axis=1)
    assert np.all(np.abs(r["lnl_inco"] - ref["lnl_inco"]) <= tol_i)
    np.testing.assert_allclose(r["lnl_inco"], r["lnl_ml"].astype(np.float64).sum(axis=1), rtol=0, atol=0)
    # the maximum and the window
    assert r["max_lnl_inco"] == r["lnl_inco"].max()
    assert r["threshold"] == r["max_lnl_inco"] - 20.0
    assert r["lnl_inco"][r["arg_i"]] == r["max_lnl_inco"]
    assert abs(r["max_lnl_inco"] - ref["lnl_inco"].max()) <= tol_i.max()
    keep_gpu = np.zeros(1000, bool)
    keep_gpu[r["selected"]] = True
    assert np.all(np.diff(r["selected"]) > 0)
    np.testing.assert_array_equal(keep_gpu, r["lnl_inco"] >= r["threshold"])
    clear = np.abs(ref["lnl_inco"] - ref["threshold"]) > 2 * tol_i.max()
    np.testing.assert_array_equal(keep_gpu[clear], ref["keep"][clear])
    assert r["n_selected"] == len(r["selected"]) and r["n_selected"] >= 1
    # the kernel's (o, t): the oracle's grid there is within the tolerance of the row maximum
    import oracle
    P = oracle.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, ps.pol, wl.event.psd,
                             wl.event.data, ps.t_grid, n_phi=32)
    for i in (0, 511, 999, int(r["arg_i"]), wl.event.injection["i"]):
        for k in range(3):
            g = P.grid(i, k)
            o, t = r["arg_ot"][i, k]
            assert 0 <= o < 32 and 0 <= t < 40
            assert g[o, t] >= g.max() - 2 * tol[i, k]


def test_slice_and_cache_give_identical_rows(dpx):
    """Rows computed in a slice that starts mid tile, with the slice's own mode
    overlaps, equal the same rows of a whole-bank call (which fills the bank's
    cross-term cache) and of a call served from that cache, bit for bit."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=2048, n_ext=4, n_det=2, n_modes=3, n_bins=200, seed=43)
    ps = synth.make_presel_inputs(wl, n_t=64, dt=1e-3, seed=44)
    bid = load_bank(dp, ctx, wl, ps)
    try:
        a = dp.dotpe_preselect(ctx, bid, 300, 700, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16)
        full = dp.dotpe_preselect(ctx, bid, 0, 2048, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16)
        b = dp.dotpe_preselect(ctx, bid, 300, 700, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    np.testing.assert_array_equal(a["lnl_ml"], full["lnl_ml"][300:700])
    np.testing.assert_array_equal(a["arg_ot"], full["arg_ot"][300:700])
    np.testing.assert_array_equal(b["lnl_ml"], a["lnl_ml"])
    np.testing.assert_array_equal(b["lnl_inco"], a["lnl_inco"])


def test_noiseless_injection_reaches_half_dd(dpx):
    """Data = the two polarisation templates of one row at a grid point: that
    row's ln L^ML_k is <d_k|d_k>/2 in every detector, and it is the maximum."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=384, n_ext=4, n_det=3, n_modes=4, n_bins=256, seed=45)
    ps = synth.make_presel_inputs(wl, n_t=32, dt=1e-3, seed=46)
    rng = np.random.default_rng(47)
    i_star, o_star, n_phi = 200, 5, 32
    data = np.zeros_like(wl.event.data)
    half_dd = []
    for k in range(3):
        t_star = 3 + 7 * k
        phi = 2 * np.pi * o_star / n_phi
        shift = np.exp(-2j * np.pi * wl.bank.f * ps.t_grid[k, t_star])
        for q in range(2):
            tpl = sum(ps.pol[i_star, m, q] * wl.bank.h[i_star, m] * np.exp(1j * wl.bank.mode_m[m] * phi)
                      for m in range(4)) * shift
            data[k] += rng.uniform(2.0, 6.0) * tpl
        half_dd.append(0.5 * np.sum(4 * wl.bank.w * np.abs(data[k]) ** 2 / wl.event.psd[k]))
    bid = load_bank(dp, ctx, wl, ps)
    try:
        r = dp.dotpe_preselect(ctx, bid, 0, 384, wl.event.psd, data, ps.t_grid, n_phi=n_phi)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    for k in range(3):
        assert r["lnl_ml"][i_star, k] == pytest.approx(half_dd[k], abs=split_tol(half_dd[k]))
        assert tuple(r["arg_ot"][i_star, k]) == (o_star, 3 + 7 * k)
    assert r["arg_i"] == i_star


def test_paper_scale_sampled_rows_against_oracle(dpx):
    """65,536 rows, 3 detectors, 4 modes, 512 bins, N_t = 128, N_phi = 32 (the
    scale of Table flops): sampled rows, the maximum and the injected row
    against the oracle; the selection window is self-consistent and keeps the
    injected row."""
    dp, ctx = dpx
    wl = synth.named_workload("cfg2")
    ps = synth.make_presel_inputs(wl)
    bid = load_bank(dp, ctx, wl, ps)
    try:
        r = dp.dotpe_preselect(ctx, bid, 0, 65536, wl.event.psd, wl.event.data, ps.t_grid, n_phi=32)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    rng = np.random.default_rng(48)
    inj = wl.event.injection["i"]
    rows = np.unique(np.concatenate([rng.choice(65536, 200, replace=False), [inj, r["arg_i"], 0, 65535]]))
    _, ref = oracle_rows(wl, ps, rows, 32)
    tol = split_tol(ref["ml"])
    d = np.abs(r["lnl_ml"][rows] - ref["ml"])
    print(f"presel 65536 rows fp16x3: max |d ln L^ML_ik| {d.max():.3e}, "
          f"kernel {r['kernel_ms']:.3f} ms, call {r['device_ms']:.3f} ms, kept {r['n_selected']}")
    assert np.all(d <= tol), float(d.max())
    keep = np.zeros(65536, bool)
    keep[r["selected"]] = True
    np.testing.assert_array_equal(keep, r["lnl_inco"] >= r["max_lnl_inco"] - 20.0)
    assert keep[inj]
    assert 1 <= r["n_selected"] < 65536


def test_invalid_requests_are_rejected(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=256, n_ext=2, n_det=2, n_modes=3, n_bins=64, seed=49)
    ps = synth.make_presel_inputs(wl, n_t=8, dt=1e-3)
    nopol = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m)
    bid = load_bank(dp, ctx, wl, ps)
    try:
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_preselect(ctx, nopol, 0, 256, wl.event.psd, wl.event.data, ps.t_grid)
        assert ei.value.status == dp.DOTPE_E_INVALID and "pol" in str(ei.value)
        for kw in (dict(n_phi=33), dict(precision="fp32"), dict(precision="mixed"), dict(delta=-1.0)):
            with pytest.raises(dp.DotpeError) as ei:
                dp.dotpe_preselect(ctx, bid, 0, 256, wl.event.psd, wl.event.data, ps.t_grid, **kw)
            assert ei.value.status == dp.DOTPE_E_INVALID
        with pytest.raises(dp.DotpeError):
            dp.dotpe_preselect(ctx, bid, 0, 257, wl.event.psd, wl.event.data, ps.t_grid)
        bad = wl.event.data.copy()
        bad[1, 3] = np.nan
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_preselect(ctx, bid, 0, 256, wl.event.psd, bad, ps.t_grid)
        assert ei.value.status == dp.DOTPE_E_INVALID
        # the context still serves after the rejections
        r = dp.dotpe_preselect(ctx, bid, 0, 256, wl.event.psd, wl.event.data, ps.t_grid)
        assert r["n_selected"] >= 1
    finally:
        dp.dotpe_bank_release(ctx, nopol)
        dp.dotpe_bank_release(ctx, bid)


# ---------------------------------------------------------------------------
# polarisation-resolved (precessing) bank: App. B with the bank's own h_imp
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def presw():
    import oracle
    wl = synth.make_precessing_workload(700, 4, 3, 4, 256, snr=15.0, seed=45, n_phi=32)
    n_t = 150
    t_grid = np.tile((np.arange(n_t) - n_t // 2) * 5e-4, (3, 1))
    P = oracle.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, None, wl.event.psd, wl.event.data,
                             t_grid, n_phi=32)
    return wl, t_grid, P, P.run(delta=20.0)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "bf16x3", "fp16"])
def test_polarisation_resolved_bank(dpx, presw, precision):
    """All rows of a 700-row precessing bank (a ragged row block), 150 times
    (FP32: two passes of its 128 time slots; tensor cores: 32-column tiles of
    the (time, polarisation, part) operand rows), against the oracle: the split
    bound 2e-3 + 1e-4 ln L^ML (FP32 and the split precisions; K = 4B here),
    the single-pass bound for fp16; the (o, t) within it; the kept set away
    from the threshold; a slice equals the whole-bank call (the slice's own
    records against the bank's cached ones)."""
    dp, ctx = dpx
    wl, t_grid, P, ref = presw
    n_t = t_grid.shape[1]
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        part = dp.dotpe_preselect(ctx, bid, 150, 250, wl.event.psd, wl.event.data, t_grid, n_phi=32, delta=20.0,
                                  precision=precision)
        r = dp.dotpe_preselect(ctx, bid, 0, 700, wl.event.psd, wl.event.data, t_grid, n_phi=32, delta=20.0,
                               precision=precision)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    assert r["device_status"] == 0
    ml_ref = ref["ml"]
    tol = fp16_tol(ml_ref, dd_per_detector(wl)[None, :]) if precision == "fp16" else split_tol(ml_ref)
    d = np.abs(r["lnl_ml"] - ml_ref)
    print(f"presel precessing {precision}: max |d ln L^ML_ik| {d.max():.3e} (ln L^ML up to {ml_ref.max():.1f})")
    assert np.all(d <= tol)
    tol_i = tol.sum(axis=1)
    assert np.all(np.abs(r["lnl_inco"] - ref["lnl_inco"]) <= tol_i)
    keep_gpu = np.zeros(700, bool)
    keep_gpu[r["selected"]] = True
    clear = np.abs(ref["lnl_inco"] - ref["threshold"]) > 2 * tol_i.max()
    np.testing.assert_array_equal(keep_gpu[clear], ref["keep"][clear])
    for i in (0, 350, 699, int(r["arg_i"]), wl.event.injection["i"]):
        for k in range(3):
            g = P.grid(i, k)
            o, t = r["arg_ot"][i, k]
            assert 0 <= o < 32 and 0 <= t < n_t
            assert g[o, t] >= g.max() - 2 * tol[i, k]
    np.testing.assert_array_equal(part["lnl_ml"], r["lnl_ml"][150:250])
    np.testing.assert_array_equal(part["arg_ot"], r["arg_ot"][150:250])


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
def test_long_bin_axis(dpx, precision):
    """B = 2,000 bins (K = 4,000: 63 k-blocks, an odd count), two detectors,
    two modes, 20 times, 200 rows: every row against the oracle."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=200, n_ext=4, n_det=2, n_modes=2, n_bins=2000, seed=47, snr=15.0)
    ps = synth.make_presel_inputs(wl, n_t=20, dt=1e-3, seed=48)
    _, ref = oracle_rows(wl, ps, np.arange(200), 16)
    bid = load_bank(dp, ctx, wl, ps)
    try:
        r = dp.dotpe_preselect(ctx, bid, 0, 200, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16, delta=20.0,
                               precision=precision)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    d = np.abs(r["lnl_ml"] - ref["ml"])
    print(f"presel B=2000 {precision}: max |d ln L^ML_ik| {d.max():.3e} (ln L^ML up to {ref['ml'].max():.1f})")
    assert np.all(d <= split_tol(ref["ml"]))


@pytest.mark.parametrize("shape", [(1, 1, 1, 1, 1), (3, 2, 2, 3, 3), (4, 3, 3, 2, 4), (5, 2, 4, 5, 12),
                                   (70, 2, 4, 3, 24)])
@pytest.mark.parametrize("bank", ["modes", "precessing"])
def test_degenerate_preselection(dpx, shape, bank):
    """Tiny shapes: one row, one detector, one mode, one time and one phase;
    three rows, two detectors and modes, three times and three phases (no
    phase pairing); 4 and 12 phases (an odd number of quarter-turn base
    phases) and 24 phases over 70 rows (base phases in pairs, a ragged second
    row tile), for a mode bank (fp16x3) and a polarisation-resolved bank
    (fp16x3 and FP32), against the oracle."""
    dp, ctx = dpx
    import oracle
    I, D, M, NT, NPH = shape
    if bank == "modes":
        wl = synth.make_workload(n_int=I, n_ext=2, n_det=D, n_modes=M, n_bins=48, seed=95, snr=12.0)
        ps = synth.make_presel_inputs(wl, n_t=NT, dt=1e-3, seed=96)
        pol, t_grid, precs = ps.pol, ps.t_grid, ("fp16x3",)
    else:
        wl = synth.make_precessing_workload(I, 2, D, M, 48, snr=12.0, seed=97, n_phi=NPH)
        pol, t_grid, precs = None, np.tile((np.arange(NT) - NT // 2) * 1e-3, (D, 1)), ("fp16x3", "fp32")
    P = oracle.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, pol, wl.event.psd, wl.event.data,
                             t_grid, n_phi=NPH)
    ref = P.run(delta=20.0)
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w, pol=pol)
    try:
        for prec in precs:
            r = dp.dotpe_preselect(ctx, bid, 0, I, wl.event.psd, wl.event.data, t_grid, n_phi=NPH, delta=20.0,
                                   precision=prec)
            assert np.all(np.abs(r["lnl_ml"] - ref["ml"]) <= split_tol(ref["ml"])), prec
            assert r["n_selected"] == int(ref["keep"].sum()) or I > 1
    finally:
        dp.dotpe_bank_release(ctx, bid)
