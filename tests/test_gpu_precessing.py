"""Polarisation-resolved (precessing) banks on the device, through the C ABI,
against the FP64 oracle (Sec. IV.A general case: Eqs. dh_ieo and hh_ieo with
the polarisation index p and real antenna patterns F_{edp}).

* An FP32 event over the whole bank (cross terms from the per-bank cache), a
  slice of it (cross terms per slice), and the whole bank streamed in blocks of
  256 rows (256, 256, 128) each meet the coherent path's FP32 tolerances against the oracle's
  route O2, all pairs: 1e-3 per pair in ln Lbar and max_o ln L^ML, 1e-2 in ln Z.
* Recomputed blocks (dotpe_lnl_blocks without stored values) read the same
  antenna patterns.
* The tensor-core precisions (K = 4B: both polarisations' real and imaginary
  parts) meet the mode bank's bounds: split fp16x3 / bf16x3 1e-3 per pair;
  single-pass fp16 2e-2 + 4u ln L^ML + 2u sqrt(2 ln L^ML + 1)
  sqrt(<d|d>); mixed the split bound within 30 of the maximum and the fp16 bound
  elsewhere; |d ln Z| <= 1e-2 for the split and mixed precisions.
* Posterior samples (dotpe_posterior_samples, the pair recomputed per (mode,
  polarisation) component) match the oracle's resampling with the same
  uniforms: identical (i, e, o) except within the weights' tolerance of a
  cumulative boundary, distances to 2e-3.
* Pre-selection with relative binning and batches in a tensor-core precision
  are refused with DOTPE_E_UNSUPPORTED; a missing F with DOTPE_E_INVALID.
  (Relative binning of events with component weights is tested with the other
  relative-binning cases, the pre-selection of such banks with the other
  pre-selection cases.)
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dpx():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    ctx = dp.dotpe_create(0)
    yield dp, ctx
    dp.dotpe_destroy(ctx)


@pytest.fixture(scope="module")
def pwl():
    import oracle
    # 640 rows (5 row tiles), 200 samples (a ragged column tile), 3 detectors, 4 modes
    wl = synth.make_precessing_workload(640, 200, 3, 4, 256, snr=18.0, seed=61, n_phi=32, ln_w="random")
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    return wl, P, grid


def run_event(dp, ctx, bid, wl, i0, i1, flags, block_rows=0):
    eid = dp.dotpe_event_submit(ctx, bid, i0, i1, wl.event.psd, wl.event.data, wl.ext.t, None, wl.ext.ln_w,
                                n_phi=wl.event.n_phi, u_min=wl.event.u_min, cut_delta=0.0, precision="fp32",
                                flags=flags, block_rows=block_rows, F=wl.ext.F)
    dp.dotpe_event_wait(ctx, eid, 120.0)
    E = wl.ext.t.shape[0]
    ev = dp.dotpe_evidence(ctx, eid)
    lnl = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E)
    ml = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E, what=dp.DOTPE_LNL_ML_MAX)
    dp.dotpe_event_release(ctx, eid)
    return ev, lnl, ml


@pytest.mark.parametrize("case", ["whole", "slice", "blocks", "recompute"])
def test_event_against_oracle(dpx, pwl, case):
    dp, ctx = dpx
    import oracle
    wl, P, grid = pwl
    bank = wl.bank
    I = bank.h.shape[0]
    i0, i1 = (0, I) if case in ("whole", "recompute", "blocks") else (128, 256)
    flags = 0 if case == "recompute" else dp.DOTPE_FLAG_STORE_LNL
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        ev, lnl, ml = run_event(dp, ctx, bid, wl, i0, i1, flags, 256 if case == "blocks" else 0)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    sub = grid[i0:i1]
    if i0 or i1 != I:
        sbank = synth.Bank(**{**bank.__dict__, "h": bank.h[i0:i1], "ln_w": bank.ln_w[i0:i1]})
        P = oracle.OracleProblem(sbank, wl.ext, wl.event)
    ref = P.evidence(sub)
    d1 = np.abs(lnl - sub["lnl_marg"])
    d2 = np.abs(ml - sub["lnl_ml_max"])
    print(f"precessing {case}: max |d ln Lbar| {d1.max():.3e}, max |d ln L^ML| {d2.max():.3e}, "
          f"d ln Z {ev['ln_z'] - ref['ln_z']:.3e}, peak ln L^ML {sub['lnl_ml_max'].max():.1f}")
    assert np.all(d1 <= 1e-3)
    assert np.all(d2 <= 1e-3)
    assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2
    assert (ev["arg_i"], ev["arg_e"]) == (i0 + ref["arg"][0], ref["arg"][1])  # arg_i is a bank row


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3", "mixed", "fp16"])
def test_tensor_core_precisions(dpx, pwl, precision):
    dp, ctx = dpx
    wl, P, grid = pwl
    bank = wl.bank
    I, B = bank.h.shape[0], bank.h.shape[-1]
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t, None, wl.ext.ln_w,
                                    n_phi=wl.event.n_phi, u_min=wl.event.u_min, cut_delta=0.0,
                                    precision=precision, flags=dp.DOTPE_FLAG_STORE_LNL, F=wl.ext.F)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        E = wl.ext.t.shape[0]
        ev = dp.dotpe_evidence(ctx, eid)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E)
        ml = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E, what=dp.DOTPE_LNL_ML_MAX)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    ref = P.evidence(grid)
    ml_ref = grid["lnl_ml_max"]
    mlp = np.maximum(ml_ref, 0.0)
    u = 2.0 ** -11
    dd = float(np.sum(4 * bank.w[None, :] * np.abs(wl.event.data) ** 2 / wl.event.psd))
    split_tol = np.full_like(mlp, 1e-3)
    fp16_tol = 2e-2 + 4 * u * mlp + 2 * u * np.sqrt(2 * mlp + 1) * np.sqrt(dd)
    if precision == "fp16":
        tol = fp16_tol
    elif precision == "mixed":
        tol = np.where(ml_ref >= ml_ref.max() - 30.0, split_tol, fp16_tol)
    else:
        tol = split_tol
    d1 = np.abs(lnl - grid["lnl_marg"])
    d2 = np.abs(ml - ml_ref)
    print(f"precessing {precision}: max |d ln Lbar| {d1.max():.3e}, max |d ln L^ML| {d2.max():.3e}, "
          f"d ln Z {ev['ln_z'] - ref['ln_z']:.3e}")
    assert np.all(d1 <= tol)
    assert np.all(d2 <= tol)
    if precision != "fp16":
        assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2
        assert (ev["arg_i"], ev["arg_e"]) == ref["arg"][:2]


@pytest.mark.parametrize("shape", [(300, 77, 2, 3, 128), (129, 33, 1, 1, 96), (200, 50, 3, 2, 200),
                                   (140, 36, 2, 2, 1000)])
@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "mixed"])
def test_ragged_shapes_and_networks(dpx, shape, precision):
    """Ragged row and sample tiles, one to three detectors, one to three modes,
    and K = 4B = 800 (13 k-blocks: an odd last k-block) against the oracle."""
    dp, ctx = dpx
    import oracle
    I, E, D, M, B = shape
    wl = synth.make_precessing_workload(I, E, D, M, B, snr=14.0, seed=71 + I, n_phi=32, ln_w="random")
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ref = P.evidence(grid)
    bank = wl.bank
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t, None, wl.ext.ln_w,
                                    n_phi=32, u_min=wl.event.u_min, cut_delta=0.0, precision=precision,
                                    flags=dp.DOTPE_FLAG_STORE_LNL, F=wl.ext.F)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        ev = dp.dotpe_evidence(ctx, eid)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E)
        ml = dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E, what=dp.DOTPE_LNL_ML_MAX)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    ml_ref = grid["lnl_ml_max"]
    mlp = np.maximum(ml_ref, 0.0)
    split_tol = np.full_like(mlp, 1e-3)
    if precision == "mixed":
        u = 2.0 ** -11
        dd = float(np.sum(4 * bank.w[None, :] * np.abs(wl.event.data) ** 2 / wl.event.psd))
        tol = np.where(ml_ref >= ml_ref.max() - 30.0, split_tol,
                       2e-2 + 4 * u * mlp + 2 * u * np.sqrt(2 * mlp + 1) * np.sqrt(dd))
    elif precision == "fp16x3":
        tol = split_tol
    else:
        tol = np.full_like(ml_ref, 1e-3)
    assert np.all(np.abs(lnl - grid["lnl_marg"]) <= tol)
    assert np.all(np.abs(ml - ml_ref) <= tol)
    assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2
    assert (ev["arg_i"], ev["arg_e"]) == ref["arg"][:2]


def near_boundary(lnw, u, a, b, tol=2e-3):
    """u lies within tol (relative) of the cumulative boundary between indices
    a and b of the weights exp(lnw)."""
    p = np.exp(lnw - np.max(lnw))
    c = np.cumsum(p) / np.sum(p)
    k = min(a, b)
    return abs(c[k] - u) <= tol * max(1.0, c[k])


@pytest.mark.parametrize("cut", [0.0, 20.0])
def test_posterior_samples_against_oracle(dpx, pwl, cut):
    dp, ctx = dpx
    import oracle
    wl, P, _ = pwl
    bank = wl.bank
    I, E = bank.h.shape[0], wl.ext.t.shape[0]
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t, None, wl.ext.ln_w,
                                    n_phi=wl.event.n_phi, u_min=wl.event.u_min, cut_delta=cut, precision="fp32",
                                    flags=dp.DOTPE_FLAG_STORE_LNL, F=wl.ext.F)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        ev = dp.dotpe_evidence(ctx, eid)
        uni = np.random.default_rng(62).random((300, 4))
        gi, ge_, go, gd = dp.dotpe_posterior_samples(ctx, eid, uni)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    thr = ev["lnl_ml_threshold"]
    pi, pe = np.divmod(np.arange(I * E), E)
    grid = P.eval_pairs(pi, pe, threshold=thr).reshape(I, E)
    oev = P.evidence(grid)
    oi, oe, oo, od = oracle.posterior_samples(P, grid, oev, uni, threshold=thr)
    same = (gi == oi) & (ge_ == oe) & (go == oo)
    for s_ in np.nonzero(~same)[0]:
        if gi[s_] != oi[s_]:
            assert near_boundary(oev["ln_p_int"], uni[s_, 0], gi[s_], oi[s_]), s_
        elif ge_[s_] != oe[s_]:
            assert near_boundary(grid[oi[s_]]["lnl_marg"] + wl.ext.ln_w, uni[s_, 1], ge_[s_], oe[s_]), s_
        else:
            z, H = P.mode_components(oi[s_], oe[s_])
            dh, hh = P.rotate_phases(z, H)
            lo = np.array([oracle.dist_marg(dh[q], hh[q], P.u_min) if oracle.lnl_ml(dh[q], hh[q]) >= thr
                           else -np.inf for q in range(P.n_phi)])
            assert near_boundary(lo, uni[s_, 2], go[s_], oo[s_]), s_
    print(f"precessing samples cut={cut}: identical (i,e,o) {same.mean():.4f}, "
          f"max distance rel diff {np.max(np.abs(gd[same] / od[same] - 1)):.2e}")
    assert same.mean() >= 0.98
    np.testing.assert_allclose(gd[same], od[same], rtol=2e-3)


def test_refusals(dpx, pwl):
    dp, ctx = dpx
    wl, _, _ = pwl
    bank = wl.bank
    I, M = bank.h.shape[0], bank.h.shape[1]
    pol = np.ones((I, M, 2), np.complex128)
    bid = dp.dotpe_bank_load(ctx, bank.h, bank.f, bank.w, bank.mode_m, bank.ln_w, pol=pol)
    try:
        spec = dict(bank_id=bid, i0=0, i1=I, psd=wl.event.psd, data=wl.event.data, t=wl.ext.t, R=None,
                    n_phi=32, u_min=wl.event.u_min, precision="mixed", F=wl.ext.F)
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_batch_submit(ctx, [spec, spec])
        assert ei.value.status == dp.DOTPE_E_UNSUPPORTED
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t, None,
                                  n_phi=32, precision="fp32")
        assert ei.value.status == dp.DOTPE_E_INVALID
        D, B = wl.event.psd.shape
        t_grid = np.zeros((D, 16))
        rb = (np.ones((D, M, B), np.complex128), np.ones((D, M, M, B), np.complex128))
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_preselect(ctx, bid, 0, I, None, None, t_grid, n_phi=32, delta=20.0, precision="fp16x3",
                               rb=rb)
        assert ei.value.status == dp.DOTPE_E_UNSUPPORTED
    finally:
        dp.dotpe_bank_release(ctx, bid)
