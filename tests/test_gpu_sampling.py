"""Posterior samples on the device (dotpe_posterior_samples) against the
oracle's resampling with the same uniforms.

The draws are discrete choices taken from cumulative weights, computed by the
device from its own (FP32-accurate) ln Lbar values and by the oracle in FP64:
a sample may land on a neighbouring index only where its uniform lies within
the weights' tolerance of a cumulative boundary.  So every sample must agree
on (i, e, o) or sit within that tolerance of the boundary between the two
choices; where (i, e, o) agree, the distances agree to 2e-3 relative.
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


def near_boundary(lnw, u, a, b, tol=2e-3):
    """The uniform u lies within tol (relative) of the cumulative boundary
    between indices a and b of the weights exp(lnw)."""
    p = np.exp(lnw - np.max(lnw))
    c = np.cumsum(p) / np.sum(p)
    k = min(a, b)
    return abs(c[k] - u) <= tol * max(1.0, c[k])


@pytest.mark.parametrize("cut", [0.0, 20.0])
def test_samples_against_oracle(dpx, cut):
    dp, ctx = dpx
    import oracle
    wl = synth.make_workload(n_int=512, n_ext=128, n_det=2, n_modes=3, n_bins=256, seed=31, snr=12.0,
                             ln_w="random")
    I, E = 512, 128
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R, wl.ext.ln_w,
                                    n_phi=wl.event.n_phi, u_min=wl.event.u_min, cut_delta=cut, precision="fp32",
                                    flags=dp.DOTPE_FLAG_STORE_LNL)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        ev = dp.dotpe_evidence(ctx, eid)
        n = max(200, int(ev["n_eff"] / 2))  # N_s = N_eff / 2 (at least 200 for the comparison)
        uni = np.random.default_rng(32).random((n, 4))
        gi, ge_, go, gd = dp.dotpe_posterior_samples(ctx, eid, uni)
        gi2, ge2, go2, gd2 = dp.dotpe_posterior_samples(ctx, eid, uni)
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    # deterministic given the uniforms
    np.testing.assert_array_equal(gi, gi2)
    np.testing.assert_array_equal(gd, gd2)
    thr = ev["lnl_ml_threshold"]
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    pi, pe = np.divmod(np.arange(I * E), E)
    grid = P.eval_pairs(pi, pe, threshold=thr).reshape(I, E)
    oev = P.evidence(grid)
    oi, oe, oo, od = oracle.posterior_samples(P, grid, oev, uni, threshold=thr)
    lw_e = wl.ext.ln_w
    same = (gi == oi) & (ge_ == oe) & (go == oo)
    for s in np.nonzero(~same)[0]:
        if gi[s] != oi[s]:
            assert near_boundary(oev["ln_p_int"], uni[s, 0], gi[s], oi[s]), s
        elif ge_[s] != oe[s]:
            assert near_boundary(grid[oi[s]]["lnl_marg"] + lw_e, uni[s, 1], ge_[s], oe[s]), s
        else:
            z, H = P.mode_components(oi[s], oe[s])
            dh, hh = P.rotate_phases(z, H)
            lo = np.array([oracle.dist_marg(dh[q], hh[q], P.u_min) if oracle.lnl_ml(dh[q], hh[q]) >= thr
                           else -np.inf for q in range(P.n_phi)])
            assert near_boundary(lo, uni[s, 2], go[s], oo[s]), s
    print(f"samples cut={cut}: n={n} (N_eff {ev['n_eff']:.0f}), identical (i,e,o) {same.mean():.4f}, "
          f"max distance rel diff {np.max(np.abs(gd[same] / od[same] - 1)):.2e}")
    assert same.mean() >= 0.98
    np.testing.assert_allclose(gd[same], od[same], rtol=2e-3)
    # the phases drawn pass the cut
    if cut > 0:
        for s in range(0, n, max(1, n // 50)):
            z, H = P.mode_components(gi[s], ge_[s])
            dh, hh = P.rotate_phases(z, H)
            assert oracle.lnl_ml(dh[go[s]], hh[go[s]]) >= thr - 1e-3


def test_samples_need_stored_values(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=128, n_ext=32, n_det=2, n_modes=3, n_bins=64, seed=33)
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, 128, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                    n_phi=wl.event.n_phi, u_min=wl.event.u_min, precision="fp32")
        dp.dotpe_event_wait(ctx, eid, 60.0)
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_posterior_samples(ctx, eid, np.full((4, 4), 0.5))
        assert ei.value.status == dp.DOTPE_E_INVALID
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
