"""The paper's two stages through the C ABI (Sec. IV.D then Sec. IV.B): the
incoherent pre-selection keeps rows, dotpe_bank_subset gathers them into a
new bank, and the coherent evaluation runs on it.

* The subset bank reproduces the parent's rows exactly: the FP32 event's
  per-pair values over the subset equal the parent event's values on the
  same rows bit for bit, and so does the pre-selection of the subset.
* The coherent result over the kept rows meets the oracle's on the same rows
  (ln Z within 1e-2, per-pair bounds of the precision).
* Bad row lists are refused.
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


def event(dp, ctx, bid, wl, n_rows, precision):
    eid = dp.dotpe_event_submit(ctx, bid, 0, n_rows, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R, wl.ext.ln_w,
                                n_phi=wl.event.n_phi, u_min=wl.event.u_min, cut_delta=0.0, precision=precision,
                                flags=dp.DOTPE_FLAG_STORE_LNL)
    dp.dotpe_event_wait(ctx, eid, 120.0)
    E = wl.ext.t.shape[0]
    out = dict(ev=dp.dotpe_evidence(ctx, eid), lnl=dp.dotpe_lnl_blocks(ctx, eid, 0, n_rows, 0, E),
               ml=dp.dotpe_lnl_blocks(ctx, eid, 0, n_rows, 0, E, what=dp.DOTPE_LNL_ML_MAX))
    dp.dotpe_event_release(ctx, eid)
    return out


def test_preselect_then_coherent_on_the_kept_rows(dpx):
    dp, ctx = dpx
    import oracle
    wl = synth.make_workload(n_int=2048, n_ext=160, n_det=3, n_modes=4, n_bins=256, seed=101, snr=15.0,
                             ln_w="random", n_phi=32)
    ps = synth.make_presel_inputs(wl, n_t=64, dt=1e-3, seed=102)
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w, pol=ps.pol)
    sub = None
    try:
        r = dp.dotpe_preselect(ctx, bid, 0, 2048, wl.event.psd, wl.event.data, ps.t_grid, n_phi=32, delta=20.0)
        kept = np.asarray(r["selected"], dtype=np.int64)
        assert 1 <= kept.size < 2048 and wl.event.injection["i"] in set(kept.tolist())
        sub = dp.dotpe_bank_subset(ctx, bid, kept)
        # the subset reproduces the parent's rows
        full = event(dp, ctx, bid, wl, 2048, "fp32")
        part = event(dp, ctx, sub, wl, kept.size, "fp32")
        np.testing.assert_array_equal(part["lnl"], full["lnl"][kept])
        np.testing.assert_array_equal(part["ml"], full["ml"][kept])
        r2 = dp.dotpe_preselect(ctx, sub, 0, kept.size, wl.event.psd, wl.event.data, ps.t_grid, n_phi=32,
                                delta=20.0)
        np.testing.assert_array_equal(r2["lnl_ml"], r["lnl_ml"][kept])
        mixed = event(dp, ctx, sub, wl, kept.size, "mixed")
        # bad row lists
        for bad in (np.array([0, 2048]), np.array([-1])):
            with pytest.raises(dp.DotpeError) as ei:
                dp.dotpe_bank_subset(ctx, bid, bad)
            assert ei.value.status == dp.DOTPE_E_INVALID
    finally:
        if sub is not None:
            dp.dotpe_bank_release(ctx, sub)
        dp.dotpe_bank_release(ctx, bid)
    # the coherent stage on the kept rows against the oracle on the same rows
    sbank = synth.Bank(**{**wl.bank.__dict__, "h": wl.bank.h[kept], "ln_w": wl.bank.ln_w[kept],
                          "mchirp": wl.bank.mchirp[kept]})
    P = oracle.OracleProblem(sbank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ref = P.evidence(grid)
    assert np.all(np.abs(part["lnl"] - grid["lnl_marg"]) <= 1e-3)
    assert abs(part["ev"]["ln_z"] - ref["ln_z"]) <= 1e-2
    assert abs(mixed["ev"]["ln_z"] - ref["ln_z"]) <= 1e-2
    assert (mixed["ev"]["arg_i"], mixed["ev"]["arg_e"]) == ref["arg"][:2]
    print(f"pipeline: kept {kept.size} of 2048 rows, ln Z {ref['ln_z']:.4f} (oracle), "
          f"fp32 {part['ev']['ln_z'] - ref['ln_z']:.2e}, mixed {mixed['ev']['ln_z'] - ref['ln_z']:.2e}")
