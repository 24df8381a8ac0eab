"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per pair, on ln Lbar_ie and max_o ln L^ML_ie):
  fp32, bf16x3, fp16x3 : |d| <= 1e-3    (the split-precision bound)
  mixed (the served path: fp16 screen + fp16x3 refinement): pairs within 30 of
         the maximum ln L^ML (which lie in refined tiles) meet 1e-3, the others
         the fp16 error model below; ln Z meets 1e-2.
  ln Z : |d| <= 1e-2 for fp32, bf16x3, fp16x3 and mixed.
Single pass (fp16, bf16: not served precisions).  A single-pass format rounds
both GEMM operands to precision u (2^-11 fp16, 2^-9 bf16), so each product
h G carries a relative error up to 2u and, by Cauchy-Schwarz,
|d<d|h>| <= 2u sqrt(<h|h><d|d>).  ln L^ML = <d|h>^2 / 2<h|h> then moves by up to
2u |x| sqrt(<d|d>) with |x| = sqrt(2 ln L^ML) (plus 4u ln L^ML when the
products add coherently).  These runs are checked against that error model,
  2e-2 + 4u ln L^ML + 2u sqrt(2 ln L^ML + 1) sqrt(<d|d>),
which is an error model and not a target: bf16 x 1 misses the flat 2e-2 per
pair (and 1e-2 in ln Z) that the target sets for BF16 at SNR 15, because the
noise power <d|d> ~ 2 B D enters every pair; test_bf16_single_pass_flat_bound
records that miss (strict xfail), and no served path runs bf16 x 1.
"""
import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {"fp32": (1e-3, 0.0), "bf16x3": (1e-3, 0.0), "fp16x3": (1e-3, 0.0), "fp16": (2e-2, 4 * 2.0 ** -11),
       "bf16": (2e-2, 4 * 2.0 ** -9), "mixed": (2e-2, 4 * 2.0 ** -11)}
PRECISE = ("fp32", "bf16x3", "fp16x3", "mixed")
MIXED_WINDOW = 30.0  # with the cut off, tiles within this of the maximum are refined


@pytest.fixture(scope="module")
def dpx():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    ctx = dp.dotpe_create(0)
    yield dp, ctx
    dp.dotpe_destroy(ctx)


def run(dp, ctx, wl, precision, bid=None, i0=0, i1=None, cut=0.0, flags=None, n_phi=None):
    own = bid is None
    if own:
        bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    I = wl.bank.h.shape[0]
    i1 = I if i1 is None else i1
    E = wl.ext.t.shape[0]
    flags = dp.DOTPE_FLAG_STORE_LNL if flags is None else flags
    eid = dp.dotpe_event_submit(ctx, bid, i0, i1, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                wl.ext.ln_w, n_phi=n_phi or wl.event.n_phi, u_min=wl.event.u_min,
                                cut_delta=cut, precision=precision, flags=flags)
    dp.dotpe_event_wait(ctx, eid, 120.0)
    ev = dp.dotpe_evidence(ctx, eid)
    out = dict(ev=ev)
    if flags & dp.DOTPE_FLAG_STORE_LNL:
        out["lnl"] = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E)
        out["ml"] = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E, what=dp.DOTPE_LNL_ML_MAX)
    out["row"] = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E, what=dp.DOTPE_ROW_MARGINAL)
    out["col"] = dp.dotpe_lnl_blocks(ctx, eid, 0, i1 - i0, 0, E, what=dp.DOTPE_COL_MARGINAL)
    out["stats"] = dp.dotpe_event_poll(ctx, eid)[1]
    dp.dotpe_event_release(ctx, eid)
    if own:
        dp.dotpe_bank_release(ctx, bid)
    return out


def data_norm(wl):
    """<d|d> = sum_d sum_b 4 w_b |d_d(f_b)|^2 / S_d(f_b) (Eq. inner_product)."""
    return float(np.sum(4.0 * wl.bank.w[None, :] * np.abs(wl.event.data) ** 2 / wl.event.psd))


def check_pairs(got, ref, precision, dd=0.0):
    a, r = TOL[precision]
    ml = np.maximum(ref["lnl_ml_max"], 0.0)
    tol = a + r * ml
    if r > 0.0:
        tol = tol + 0.5 * r * np.sqrt(2.0 * ml + 1.0) * np.sqrt(dd)
    if precision == "mixed":
        tol = np.where(ml >= ml.max() - MIXED_WINDOW, 1e-3, tol)
    d1 = np.abs(got["lnl"].astype(np.float64) - ref["lnl_marg"])
    d2 = np.abs(got["ml"].astype(np.float64) - ref["lnl_ml_max"])
    assert np.all(np.isfinite(got["lnl"]))
    assert np.all(d1 <= tol), (precision, float(d1.max()), np.unravel_index(np.argmax(d1 - tol), d1.shape))
    assert np.all(d2 <= tol), (precision, float(d2.max()))


def check_evidence(got, ref_ev, precision, lnz_tol=1e-2):
    ev = got["ev"]
    if precision in PRECISE:
        assert abs(ev["ln_z"] - ref_ev["ln_z"]) <= lnz_tol
        for k in ("n_eff", "n_eff_int", "n_eff_ext"):
            assert ev[k] == pytest.approx(ref_ev[k], rel=2e-2), k
        for key, rk in (("row", "ln_p_int"), ("col", "ln_p_ext")):
            g, r = got[key], ref_ev[rk]
            if precision == "mixed":
                # lines far below the peak keep single-pass values
                near = r >= r.max() - 20.0
                np.testing.assert_allclose(g[near], r[near], atol=2e-3)
                np.testing.assert_allclose(g, r, atol=0.2)
            else:
                np.testing.assert_allclose(g, r, atol=2e-3)
    else:
        assert abs(ev["ln_z"] - ref_ev["ln_z"]) <= 0.1


# ---------------------------------------------------------------------------
# device distance marginal (Eq. lnl_dist_marginalized) against the oracle
# ---------------------------------------------------------------------------
def test_dist_marg_table_sweep(dpx):
    """Bound: 1e-4 for the table, plus the conditioning of FP32 inputs: x = dh/sqrt(hh)
    carries ~2^-22 relative error and d lnLbar/dx lies between s and max(x, s)."""
    import oracle
    dp, ctx = dpx
    rng = np.random.default_rng(0)
    for u_min in (0.5, 2.0, 9.5):
        x = np.concatenate([rng.uniform(-60, 60, 2500), rng.uniform(0.0, 12.0, 1000)])
        s = np.exp(np.concatenate([rng.uniform(-11, 4.5, 2500), rng.uniform(-11.5, -3.0, 1000)]))
        x[2500:] += s[2500:]  # the small-s corner with y = x - s in [0, 12]
        hh = (s / u_min) ** 2
        dh = (x * np.sqrt(hh)).astype(np.float32)
        hh = hh.astype(np.float32)
        got = dp.dotpe_dist_marg_eval(ctx, dh, hh, u_min).astype(np.float64)
        ref = np.array([oracle.dist_marg(float(a), float(b), u_min) for a, b in zip(dh, hh)])
        err = np.abs(got - ref)
        bound = 1e-4 + 2.5e-7 * np.abs(x) * (np.maximum(np.abs(x), s) + 5.0) + 2e-7 * np.abs(ref)
        k = int(np.argmax(err - bound))
        assert np.all(err <= bound), (float(err[k]), float(x[k]), float(s[k]), float(ref[k]))
        assert np.median(err) < 2e-5
    # no signal power -> exactly 0
    z = dp.dotpe_dist_marg_eval(ctx, np.array([0.3, 0.0], np.float32), np.array([0.0, 0.0], np.float32), 2.0)
    assert np.all(z == 0.0)


# ---------------------------------------------------------------------------
# config 1 (all pairs): I=1024, E=256, D=2, M=3, B=256, SNR 15, seed 0
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg1():
    import oracle
    wl = synth.named_workload("cfg1", ln_w="random")
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    return wl, P, grid, P.evidence(grid)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16x3", "mixed", "fp16", "bf16"])
def test_config1_all_pairs(dpx, cfg1, precision):
    dp, ctx = dpx
    wl, P, grid, ref_ev = cfg1
    got = run(dp, ctx, wl, precision)
    check_pairs(got, grid, precision, data_norm(wl))
    check_evidence(got, ref_ev, precision)
    if precision in PRECISE:
        assert (got["ev"]["arg_i"], got["ev"]["arg_e"], got["ev"]["arg_o"]) == tuple(ref_ev["arg"])
        assert got["ev"]["max_lnl_ml"] == pytest.approx(ref_ev["max_lnl_ml"], abs=1e-3)
    assert got["ev"]["n_marginalised"] == ref_ev["n_marginalised"]


@pytest.mark.xfail(strict=True, reason="single-pass bf16 misses the flat 2e-2 per pair and 1e-2 in ln Z at "
                                       "SNR 15 (operand rounding 2^-9 against <d|d> ~ 2 B D); not a served "
                                       "precision")
def test_bf16_single_pass_flat_bound(dpx, cfg1):
    """The target's flat BF16 bound, |d ln L| <= 2e-2 per pair and |d ln Z| <= 1e-2,
    applied to bf16 x 1 at configuration 1: expected to fail (see the module
    docstring); the split and mixed paths are the ones that meet their bounds."""
    dp, ctx = dpx
    wl, P, grid, ref_ev = cfg1
    got = run(dp, ctx, wl, "bf16")
    d1 = np.abs(got["lnl"].astype(np.float64) - grid["lnl_marg"])
    d2 = np.abs(got["ml"].astype(np.float64) - grid["lnl_ml_max"])
    print(f"bf16 x 1 at configuration 1: max |d ln Lbar| {d1.max():.3e}, max |d ln L^ML| {d2.max():.3e}, "
          f"|d ln Z| {abs(got['ev']['ln_z'] - ref_ev['ln_z']):.3e}")
    assert d1.max() <= 2e-2 and d2.max() <= 2e-2
    assert abs(got["ev"]["ln_z"] - ref_ev["ln_z"]) <= 1e-2


def test_config1_ml_cut(dpx, cfg1):
    """Eq. coherent_ML_selection with the paper's delta = 20.  The device uses a
    running maximum, so it keeps a superset of the exact cut: its ln Z lies
    between the oracle's cut and uncut values."""
    import oracle
    dp, ctx = dpx
    wl, P, grid, ref_ev = cfg1
    gcut, thr = P.eval_grid(20.0)
    ev_cut = P.evidence(gcut)
    for precision in PRECISE:
        got = run(dp, ctx, wl, precision, cut=20.0, flags=0)
        ev = got["ev"]
        assert ev_cut["ln_z"] - 1e-2 <= ev["ln_z"] <= ref_ev["ln_z"] + 1e-2
        assert ev["n_marginalised"] >= ev_cut["n_marginalised"]
        assert ev["lnl_ml_threshold"] <= thr + 1e-3
        assert (ev["arg_i"], ev["arg_e"], ev["arg_o"]) == tuple(ref_ev["arg"])
        assert ev["max_lnl_ml"] == pytest.approx(ref_ev["max_lnl_ml"], abs=1e-3)
        if precision == "mixed":
            # the frozen threshold lies at most two margins below the exact one
            assert thr - 3.0 <= ev["lnl_ml_threshold"] <= thr + 1e-3
            assert 0 < ev["n_refined_tiles"] < (1024 // 128) * (256 // 32)
            # the screen's counters: every pair whose exact ln L^ML reaches the final
            # threshold passes its first bound (bounds never fall below ln L^ML, the
            # threshold only rises to it), and it evaluates a subset of what passes
            above = int(np.sum(gcut["lnl_ml_max"] >= ev["lnl_ml_threshold"] + 1e-3))
            assert above <= ev["n_screen_candidates"] <= ev["n_pairs"]
            assert 1 <= ev["n_screen_evaluated"] <= ev["n_screen_candidates"]
        else:
            assert ev["n_refined_tiles"] == -1
            assert ev["n_screen_candidates"] == -1 and ev["n_screen_evaluated"] == -1


# ---------------------------------------------------------------------------
# ragged shapes, slices, mode/detector counts
# ---------------------------------------------------------------------------
SHAPES = [  # I_bank, slice, E, D, M, B
    (200, (0, 200), 45, 1, 1, 64),
    (400, (17, 350), 77, 2, 3, 96),
    (300, (5, 134), 33, 3, 4, 160),
    (150, (0, 150), 130, 3, 2, 40),
    (140, (3, 140), 40, 2, 2, 2000),  # K = 4,000 -> 63 k-blocks of 64 (an odd count: a half-empty last box)
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"I{s[0]}E{s[2]}D{s[3]}M{s[4]}B{s[5]}")
@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "fp16x3", "mixed", "fp16", "bf16"])
def test_ragged_shapes(dpx, shape, precision):
    import oracle
    dp, ctx = dpx
    Ib, (a, b), E, D, M, B = shape
    wl = synth.make_workload(n_int=Ib, n_ext=E, n_det=D, n_modes=M, n_bins=B, snr=12.0,
                             seed=Ib + E + D, ln_w="random", n_phi=16)
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event, i_slice=slice(a, b))
    grid, _ = P.eval_grid(0.0)
    ref_ev = P.evidence(grid)
    got = run(dp, ctx, wl, precision, i0=a, i1=b)
    check_pairs(got, grid, precision, data_norm(wl))
    check_evidence(got, ref_ev, precision)
    if precision in PRECISE:
        assert got["ev"]["arg_i"] - a == ref_ev["arg"][0]
        assert (got["ev"]["arg_e"], got["ev"]["arg_o"]) == tuple(ref_ev["arg"][1:])


@pytest.mark.parametrize("case", ["one_pair_one_phase", "odd_phase_grid", "zero_data"])
@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "mixed"])
def test_degenerate_cases(dpx, case, precision):
    """Degenerate inputs against the oracle: a single (i, e) pair with one
    detector, one mode and N_phi = 1; an odd phase grid (N_phi = 7: no (phi,
    phi + pi) pairing); data identically zero (every <d|h> = 0, so ln L^ML = 0,
    ln Lbar is the distance marginal at dh = 0 and ln Z <= 0)."""
    import oracle
    dp, ctx = dpx
    if case == "one_pair_one_phase":
        wl = synth.make_workload(n_int=1, n_ext=1, n_det=1, n_modes=1, n_bins=16, snr=10.0, seed=81, n_phi=1)
    elif case == "odd_phase_grid":
        wl = synth.make_workload(n_int=130, n_ext=33, n_det=2, n_modes=3, n_bins=64, snr=12.0, seed=82, n_phi=7)
    else:
        wl = synth.make_workload(n_int=140, n_ext=40, n_det=2, n_modes=4, n_bins=64, snr=12.0, seed=83, n_phi=8)
        wl.event.data[:] = 0.0
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ref_ev = P.evidence(grid)
    got = run(dp, ctx, wl, precision)
    check_pairs(got, grid, precision, data_norm(wl))
    assert abs(got["ev"]["ln_z"] - ref_ev["ln_z"]) <= 1e-2
    if case == "zero_data":
        assert got["ev"]["ln_z"] <= 1e-6
        assert np.all(got["ml"] == 0.0)


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "mixed"])
def test_ragged_block_streaming(dpx, precision):
    """A 680-row slice streamed in 256-row blocks (256, 256, 168) against the
    oracle, all pairs, cut off (block streaming then changes nothing but FP64
    rounding); with the cut on, ln Z and the maximum equal the one-pass run's."""
    import oracle
    dp, ctx = dpx
    wl = synth.make_workload(n_int=700, n_ext=70, n_det=3, n_modes=4, n_bins=128, snr=14.0, seed=91,
                             ln_w="random", n_phi=16)
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event, i_slice=slice(20, 700))
    grid, _ = P.eval_grid(0.0)
    ref_ev = P.evidence(grid)
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        out = {}
        for cut, br in ((0.0, 256), (20.0, 256), (20.0, 0)):
            eid = dp.dotpe_event_submit(ctx, bid, 20, 700, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                        wl.ext.ln_w, n_phi=16, u_min=wl.event.u_min, cut_delta=cut,
                                        precision=precision, flags=dp.DOTPE_FLAG_STORE_LNL, block_rows=br)
            dp.dotpe_event_wait(ctx, eid, 120.0)
            out[(cut, br)] = dict(ev=dp.dotpe_evidence(ctx, eid),
                                  lnl=dp.dotpe_lnl_blocks(ctx, eid, 0, 680, 0, 70),
                                  ml=dp.dotpe_lnl_blocks(ctx, eid, 0, 680, 0, 70, what=dp.DOTPE_LNL_ML_MAX))
            dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)
    got = out[(0.0, 256)]
    check_pairs(got, grid, precision, data_norm(wl))
    assert abs(got["ev"]["ln_z"] - ref_ev["ln_z"]) <= 1e-2
    assert got["ev"]["arg_i"] - 20 == ref_ev["arg"][0]
    a, b = out[(20.0, 256)]["ev"], out[(20.0, 0)]["ev"]
    assert abs(a["ln_z"] - b["ln_z"]) <= 1e-3
    assert a["max_lnl_ml"] == b["max_lnl_ml"] and (a["arg_i"], a["arg_e"], a["arg_o"]) == (b["arg_i"], b["arg_e"], b["arg_o"])


def test_noiseless_peak(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=500, n_ext=96, n_det=3, n_modes=4, n_bins=128, snr=15.0, seed=5,
                             noise=False, insert_injection=True, phi_inj=2 * np.pi * 5 / 32)
    for precision in PRECISE:
        ev = run(dp, ctx, wl, precision, flags=0)["ev"]
        assert (ev["arg_i"], ev["arg_e"], ev["arg_o"]) == (wl.event.injection["i"], 0, 5)
        assert ev["max_lnl_ml"] == pytest.approx(112.5, abs=2e-3)


# ---------------------------------------------------------------------------
# production size (65,536 x 4,096, D=3, M=4, B=512): sampled pairs vs the oracle
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg2():
    wl = synth.named_workload("cfg2")
    return wl


def test_config2_sampled_pairs_and_evidence(dpx, cfg2):
    """Configuration 2 against the oracle on a seeded 1% (i, e) subsample
    (2,684,355 pairs, plus the peak pair), element by element, in every
    precision."""
    import oracle
    dp, ctx = dpx
    wl = cfg2
    I, E = wl.bank.h.shape[0], wl.ext.t.shape[0]
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        pi, pe = synth.pair_subsample(2, I, E, frac=0.01)
        assert pi.shape[0] == round(0.01 * I * E)
        # include the best pairs: the oracle's max must agree where it matters most
        P = oracle.OracleProblem(wl.bank, wl.ext, wl.event)
        res = {}
        for precision in ("fp32", "bf16x3", "fp16x3", "bf16", "mixed"):
            got = run(dp, ctx, wl, precision, bid=bid)
            if precision == "fp32":
                i_s, e_s = got["ev"]["arg_i"], got["ev"]["arg_e"]
                pi = np.concatenate([pi, [i_s]])
                pe = np.concatenate([pe, [e_s]])
            # keep the sampled pairs only (the full [I][E] arrays are 1 GB each)
            if precision == "bf16x3":
                got["lnl_full"] = got["lnl"]
            else:
                got["lnl"] = got["lnl"][pi, pe]
                got["ml"] = got["ml"][pi, pe]
            res[precision] = got
        ref = P.eval_pairs(pi, pe)
        for precision, got in res.items():
            if precision == "bf16x3":
                sub = {"lnl": got["lnl"][pi, pe], "ml": got["ml"][pi, pe]}
            else:
                sub = {"lnl": got["lnl"], "ml": got["ml"]}
            check_pairs(sub, ref, precision, data_norm(wl))
            if precision in ("fp32", "bf16x3", "fp16x3", "mixed"):
                d = np.abs(sub["ml"].astype(np.float64) - ref["lnl_ml_max"])
                print(f"config 2 {precision}: {pi.shape[0]} pairs, max |d ln L^ML| {d.max():.2e}")
        # evidence: served split precision against the plain FP32 path (same GPU)
        assert abs(res["bf16x3"]["ev"]["ln_z"] - res["fp32"]["ev"]["ln_z"]) <= 1e-2
        assert abs(res["mixed"]["ev"]["ln_z"] - res["fp32"]["ev"]["ln_z"]) <= 1e-2
        assert abs(res["fp16x3"]["ev"]["ln_z"] - res["fp32"]["ev"]["ln_z"]) <= 1e-2
        # the FP64 reduction reproduces a direct FP64 log-sum-exp of the stored ln Lbar_ie
        lnl = res["bf16x3"]["lnl_full"].astype(np.float64)
        lw = wl.bank.ln_w[:, None] + wl.ext.ln_w[None, :]
        x = (lnl + lw).ravel()
        m = x.max()
        lnz = m + math.log(np.sum(np.exp(x - m))) - math.log(I * E)
        assert res["bf16x3"]["ev"]["ln_z"] == pytest.approx(lnz, abs=1e-4)
        assert res["bf16x3"]["ev"]["max_lnl_ml"] == pytest.approx(float(ref["lnl_ml_max"][-1]), abs=1e-3)
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_config2_mixed_with_cut(dpx, cfg2):
    """The served path with the paper's cut (delta = 20) against the plain FP32
    path with the same cut: ln Z, the maximum and its location."""
    dp, ctx = dpx
    wl = cfg2
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        ref = run(dp, ctx, wl, "fp32", bid=bid, cut=20.0, flags=0)["ev"]
        for precision in ("bf16x3", "mixed"):
            ev = run(dp, ctx, wl, precision, bid=bid, cut=20.0, flags=0)["ev"]
            assert abs(ev["ln_z"] - ref["ln_z"]) <= 1e-2, precision
            assert ev["max_lnl_ml"] == pytest.approx(ref["max_lnl_ml"], abs=1e-3)
            assert (ev["arg_i"], ev["arg_e"], ev["arg_o"]) == (ref["arg_i"], ref["arg_e"], ref["arg_o"])
            assert ev["n_eff"] == pytest.approx(ref["n_eff"], rel=2e-2)
        n_tiles = (65536 // 128) * (4096 // 32)
        assert 0 < ev["n_refined_tiles"] < n_tiles
    finally:
        dp.dotpe_bank_release(ctx, bid)


# ---------------------------------------------------------------------------
# runtime: concurrency, admission, failure paths
# ---------------------------------------------------------------------------
def test_concurrent_events_equal_alone(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=2048, n_ext=512, n_det=3, n_modes=4, n_bins=256, snr=12.0, seed=21)
    rng = np.random.default_rng(3)
    evs = [wl.event] + [synth.make_event(rng, wl.bank, wl.ext, 3, snr=float(s)) for s in (8, 20, 35)]
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        def submit(ev, prec, i0, i1):
            return dp.dotpe_event_submit(ctx, bid, i0, i1, ev.psd, ev.data, wl.ext.t, wl.ext.R,
                                         n_phi=32, u_min=ev.u_min, precision=prec)
        specs = [(evs[k], ("bf16x3", "fp32", "bf16x3", "fp16")[k], 64 * k, 2048 - 100 * k) for k in range(4)]
        alone = []
        for s in specs:
            eid = submit(*s)
            dp.dotpe_event_wait(ctx, eid, 60)
            alone.append(dp.dotpe_evidence(ctx, eid))
            dp.dotpe_event_release(ctx, eid)
        ids = [submit(*s) for s in specs]  # all in flight together
        for eid, a in zip(ids, alone):
            dp.dotpe_event_wait(ctx, eid, 60)
            b = dp.dotpe_evidence(ctx, eid)
            # no ML cut: fixed reduction order, so results are bitwise equal
            assert b["ln_z"] == a["ln_z"] and b["n_eff"] == a["n_eff"]
            assert (b["arg_i"], b["arg_e"], b["arg_o"]) == (a["arg_i"], a["arg_e"], a["arg_o"])
            dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_release_cancels_a_queued_event():
    """Releasing an event that still waits for a slot cancels it: it never
    runs, its id is gone, and the events around it complete normally."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    wl = synth.make_workload(n_int=1024, n_ext=128, n_det=2, n_modes=3, n_bins=128, snr=12.0, seed=25)
    ctx = dp.dotpe_create(0, n_slots=1)
    try:
        bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)

        def submit(stream=None):
            return dp.dotpe_event_submit(ctx, bid, 0, 1024, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                         n_phi=16, u_min=wl.event.u_min, precision="fp32", stream=stream)
        ref = submit()
        dp.dotpe_event_wait(ctx, ref, 60.0)
        z_ref = dp.dotpe_evidence(ctx, ref)["ln_z"]
        dp.dotpe_event_release(ctx, ref)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            torch.cuda._sleep(50_000_000)  # the first event's inputs wait behind this: it holds the slot
        a = submit(stream=s)
        b = submit()
        assert dp.dotpe_event_poll(ctx, b)[0] == dp.DOTPE_STATE_QUEUED
        dp.dotpe_event_release(ctx, b)  # cancelled before it ran
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_event_poll(ctx, b)
        assert ei.value.status == dp.DOTPE_E_NOT_FOUND
        c = submit()
        for eid in (a, c):
            dp.dotpe_event_wait(ctx, eid, 60.0)
            assert dp.dotpe_evidence(ctx, eid)["ln_z"] == z_ref
            dp.dotpe_event_release(ctx, eid)
        dp.dotpe_bank_release(ctx, bid)
    finally:
        dp.dotpe_destroy(ctx)


def test_host_threads_share_one_context(dpx):
    """Four host threads submit, wait for, read and release events on one
    context at once (the ABI's calls are thread-safe on a context); each
    thread's results equal the same events run one at a time, bit for bit."""
    import threading
    dp, ctx = dpx
    wl = synth.make_workload(n_int=1536, n_ext=256, n_det=3, n_modes=4, n_bins=256, snr=12.0, seed=23)
    rng = np.random.default_rng(4)
    evs = [synth.make_event(rng, wl.bank, wl.ext, 3, snr=float(s)) for s in (9, 14, 22, 30)]
    precs = ("fp32", "bf16x3", "fp16x3", "mixed")
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)

    def one(ev, prec):
        eid = dp.dotpe_event_submit(ctx, bid, 0, 1536, ev.psd, ev.data, wl.ext.t, wl.ext.R, n_phi=32,
                                    u_min=ev.u_min, precision=prec)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        r = dp.dotpe_evidence(ctx, eid)
        dp.dotpe_event_release(ctx, eid)
        return r

    try:
        alone = [one(evs[k], precs[k]) for k in range(4)]
        got = [[None] * 3 for _ in range(4)]
        errors = []

        def worker(k):
            try:
                for rep in range(3):
                    got[k][rep] = one(evs[k], precs[k])
            except Exception as exc:  # reported below
                errors.append(exc)

        threads = [threading.Thread(target=worker, args=(k,)) for k in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join(300)
        assert not errors, errors
        for k in range(4):
            for rep in range(3):
                b, a = got[k][rep], alone[k]
                assert b["ln_z"] == a["ln_z"] and b["n_eff"] == a["n_eff"], (k, rep)
                assert (b["arg_i"], b["arg_e"], b["arg_o"]) == (a["arg_i"], a["arg_e"], a["arg_o"])
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_served_mix_equal_alone(dpx):
    """Continuous batching: uneven events (bank slices, extrinsic counts, detector
    counts, SNR) in the served precision with the paper's cut, more events than
    slots.  Each result equals the one the event gets alone (bitwise: the
    refinement threshold is frozen and every reduction has a fixed order)."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=4096, n_ext=64, n_det=3, n_modes=4, n_bins=256, snr=12.0, seed=31)
    rng = np.random.default_rng(7)
    specs = []
    for k, (E, D, snr, a, b) in enumerate([(256, 3, 9.0, 0, 4096), (512, 2, 25.0, 100, 3000), (1024, 3, 14.0, 7, 777),
                                           (333, 2, 40.0, 2048, 4096), (700, 3, 18.0, 0, 1500)]):
        ext = synth.make_extrinsic(np.random.default_rng(100 + k), E, D, wl.bank, ln_w="random")
        ev = synth.make_event(rng, wl.bank, ext, D, snr=snr, inj_i=int(rng.integers(a, b)))
        specs.append((ext, ev, a, b))
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        def submit(ext, ev, a, b):
            return dp.dotpe_event_submit(ctx, bid, a, b, ev.psd, ev.data, ext.t, ext.R, ext.ln_w,
                                         n_phi=32, u_min=ev.u_min, cut_delta=20.0, precision="mixed")
        alone = []
        for sp in specs:
            eid = submit(*sp)
            dp.dotpe_event_wait(ctx, eid, 60)
            alone.append(dp.dotpe_evidence(ctx, eid))
            dp.dotpe_event_release(ctx, eid)
        ids = [submit(*sp) for sp in specs]
        for eid, a in zip(ids, alone):
            dp.dotpe_event_wait(ctx, eid, 60)
            b = dp.dotpe_evidence(ctx, eid)
            for key in ("ln_z", "n_eff", "n_eff_int", "n_eff_ext", "max_lnl_ml", "arg_i", "arg_e", "arg_o",
                        "n_marginalised", "n_refined_tiles", "lnl_ml_threshold"):
                assert b[key] == a[key], key
            dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_admission_by_footprint(dpx):
    import paper_2507_16022_gb300 as dp
    wl = synth.make_workload(n_int=8192, n_ext=2048, n_det=3, n_modes=4, n_bins=256, snr=12.0, seed=9)
    dp0, ctx0 = dpx
    probe = run(dp0, ctx0, wl, "bf16x3", flags=0)
    foot = probe["stats"]["footprint_bytes"]
    bank_bytes = 12 * 4 * 8192 * 512 + (1 << 20)  # FP32 master + bf16 and fp16 hi/lo planes
    ctx = dp.dotpe_create(0, hbm_budget_bytes=int(bank_bytes + 1.5 * foot), n_slots=4)
    try:
        bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m)
        # an event larger than the whole budget is refused outright
        big = synth.make_workload(n_int=8, n_ext=60000, n_det=3, n_modes=4, n_bins=256, seed=1)
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_event_submit(ctx, bid, 0, 8192, wl.event.psd, wl.event.data, big.ext.t, big.ext.R,
                                  u_min=wl.event.u_min, precision="bf16x3")
        assert ei.value.status == dp.DOTPE_E_ADMISSION
        # events that fit one at a time are queued, then admitted as memory frees, and all complete
        ids = [dp.dotpe_event_submit(ctx, bid, 0, 8192, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                     u_min=wl.event.u_min, precision="bf16x3") for _ in range(3)]
        assert dp.dotpe_event_poll(ctx, ids[2])[0] == dp.DOTPE_STATE_QUEUED
        lz = []
        for e in ids:
            dp.dotpe_event_wait(ctx, e, 60)
            lz.append(dp.dotpe_evidence(ctx, e)["ln_z"])
            dp.dotpe_event_release(ctx, e)
        assert lz[0] == lz[1] == lz[2] == probe["ev"]["ln_z"]
    finally:
        dp.dotpe_destroy(ctx)


def test_nonfinite_input_reported_and_context_survives(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=256, n_ext=64, n_det=2, n_modes=3, n_bins=64, snr=10.0, seed=4)
    psd = wl.event.psd.copy()
    psd[1, 7] = np.nan
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, 256, psd, wl.event.data, wl.ext.t, wl.ext.R,
                                    u_min=wl.event.u_min, precision="bf16x3")
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_event_wait(ctx, eid, 60)
        assert ei.value.status == dp.DOTPE_E_INVALID
        dp.dotpe_event_release(ctx, eid)
        eid = dp.dotpe_event_submit(ctx, bid, 0, 256, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                    u_min=wl.event.u_min, precision="bf16x3")
        dp.dotpe_event_wait(ctx, eid, 60)
        assert math.isfinite(dp.dotpe_evidence(ctx, eid)["ln_z"])
        dp.dotpe_event_release(ctx, eid)
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_device_wait_timeout_is_reported_and_context_survives(dpx):
    """A stage that is never signalled: the bounded mbarrier wait runs out,
    the kernel records a timeout and exits; no fault, no hang."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=512, n_ext=128, n_det=2, n_modes=3, n_bins=64, snr=10.0, seed=6)
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m)
    try:
        eid = dp.dotpe_event_submit(ctx, bid, 0, 512, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                    u_min=wl.event.u_min, precision="bf16", flags=dp.DOTPE_FLAG_TEST_STALL)
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_event_wait(ctx, eid, 60)
        assert ei.value.status == dp.DOTPE_E_TIMEOUT
        assert dp.dotpe_event_poll(ctx, eid)[0] == dp.DOTPE_STATE_FAILED
        dp.dotpe_event_release(ctx, eid)
        got = run(dp, ctx, wl, "bf16x3", bid=bid, flags=0)
        assert math.isfinite(got["ev"]["ln_z"])
    finally:
        dp.dotpe_bank_release(ctx, bid)


def test_device_resident_inputs_on_caller_stream(dpx):
    import torch
    dp, ctx = dpx
    wl = synth.make_workload(n_int=700, n_ext=90, n_det=3, n_modes=4, n_bins=128, snr=12.0, seed=8)
    host = run(dp, ctx, wl, "bf16x3", flags=0)["ev"]
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        def dev(a):
            a = np.ascontiguousarray(a)
            a = a.view(np.float64) if np.iscomplexobj(a) else a
            return torch.from_numpy(a.copy()).to("cuda", non_blocking=True)
        t, R, lw, psd, data = (dev(x) for x in (wl.ext.t, wl.ext.R, wl.ext.ln_w, wl.event.psd, wl.event.data))
    eid = dp.dotpe_event_submit(ctx, bid, 0, 700, psd, data, t, R, lw, n_phi=32, u_min=wl.event.u_min,
                                precision="bf16x3", stream=s)
    dp.dotpe_event_stream_wait(ctx, eid, s)
    s.synchronize()
    assert dp.dotpe_event_poll(ctx, eid)[0] == dp.DOTPE_STATE_DONE
    ev = dp.dotpe_evidence(ctx, eid)
    assert ev["ln_z"] == host["ln_z"]
    dp.dotpe_event_release(ctx, eid)
    dp.dotpe_bank_release(ctx, bid)


def test_lnl_blocks_recomputed_without_stored_tiles(dpx):
    """An event run without DOTPE_FLAG_STORE_LNL: dotpe_lnl_blocks recomputes the
    asked block from the kept inputs.  Without the cut it equals the stored values
    of the same event run with the flag (the same per-pair arithmetic); with the
    cut it applies the event's final threshold; in mixed precision the block is
    computed in split fp16 and meets the split tolerance against the oracle."""
    import oracle
    dp, ctx = dpx
    wl = synth.make_workload(n_int=900, n_ext=200, n_det=3, n_modes=4, n_bins=128, snr=14.0, seed=12,
                             ln_w="random")
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    a, b, e0, e1 = 130, 517, 33, 170  # a ragged block, not aligned to tiles
    try:
        def sub(precision, flags, cut):
            eid = dp.dotpe_event_submit(ctx, bid, 50, 900, wl.event.psd, wl.event.data, wl.ext.t, wl.ext.R,
                                        wl.ext.ln_w, n_phi=32, u_min=wl.event.u_min, cut_delta=cut,
                                        precision=precision, flags=flags)
            dp.dotpe_event_wait(ctx, eid, 60)
            return eid
        for precision in ("fp32", "bf16x3"):
            full = sub(precision, dp.DOTPE_FLAG_STORE_LNL, 0.0)
            bare = sub(precision, 0, 0.0)
            for what in (dp.DOTPE_LNL_MARG, dp.DOTPE_LNL_ML_MAX):
                x = dp.dotpe_lnl_blocks(ctx, full, a, b, e0, e1, what=what)
                y = dp.dotpe_lnl_blocks(ctx, bare, a, b, e0, e1, what=what)
                assert np.array_equal(x, y), (precision, what)
            dp.dotpe_event_release(ctx, full)
            dp.dotpe_event_release(ctx, bare)
        # with the cut: the final threshold, fixed
        eid = sub("bf16x3", 0, 20.0)
        ev = dp.dotpe_evidence(ctx, eid)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, a, b, e0, e1)
        ml = dp.dotpe_lnl_blocks(ctx, eid, a, b, e0, e1, what=dp.DOTPE_LNL_ML_MAX)
        assert np.all(np.isneginf(lnl) <= (ml < ev["lnl_ml_threshold"] + 1e-3))
        dp.dotpe_event_release(ctx, eid)
        # mixed: split fp16 against the oracle on the block
        eid = sub("mixed", 0, 0.0)
        lnl = dp.dotpe_lnl_blocks(ctx, eid, a, b, e0, e1).astype(np.float64)
        dp.dotpe_event_release(ctx, eid)
        P = oracle.OracleProblem(wl.bank, wl.ext, wl.event, i_slice=slice(50 + a, 50 + b))
        ii, ee = np.meshgrid(np.arange(b - a), np.arange(e0, e1), indexing="ij")
        ref = P.eval_pairs(ii.ravel(), ee.ravel())
        assert np.max(np.abs(lnl.ravel() - ref["lnl_marg"])) <= 1e-3
    finally:
        dp.dotpe_bank_release(ctx, bid)


@pytest.mark.parametrize("shape", SHAPES[:4] + [(600, (0, 600), 64 * 3 + 40, 3, 4, 256),
                                                 (2048, (0, 2048), 24 * 32 + 5, 3, 4, 128)],
                         ids=lambda s: f"I{s[0]}E{s[2]}D{s[3]}M{s[4]}B{s[5]}")
def test_screen_tile_widths_agree(dpx, shape):
    """The served path's screening pass runs in 64-sample tiles on CTA pairs by
    default, in 64-sample tiles on one CTA each under DOTPE_CONFIG_SINGLE_CTA_TILES
    and in 32-sample tiles under DOTPE_CONFIG_NARROW_TILES: all mark the same
    tiles for refinement (an odd count of 32-sample tiles leaves the last
    64-sample tile half empty, an odd count of bank tiles the last pair tile;
    the largest shape has enough tiles for the pilot tiles that the wide screen
    takes first), so the events agree, and all keep ln Z between the oracle's
    cut and uncut values (Eq. coherent_ML_selection; the largest shape against
    the plain FP32 path with the same cut)."""
    import oracle
    dp, ctx = dpx
    I_bank, (i0, i1), E, D, M, B = shape
    wl = synth.make_workload(n_int=I_bank, n_ext=E, n_det=D, n_modes=M, n_bins=B, snr=14.0, seed=I_bank + E,
                             ln_w="random")
    narrow = dp.dotpe_create(0, flags=dp.DOTPE_CONFIG_NARROW_TILES)
    single = dp.dotpe_create(0, flags=dp.DOTPE_CONFIG_SINGLE_CTA_TILES)
    try:
        res = []
        for c in (ctx, narrow, single):
            bid = dp.dotpe_bank_load(c, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
            try:
                res.append(run(dp, c, wl, "mixed", bid=bid, i0=i0, i1=i1, cut=20.0, flags=0)["ev"])
            finally:
                dp.dotpe_bank_release(c, bid)
    finally:
        dp.dotpe_destroy(narrow)
        dp.dotpe_destroy(single)
    wide, nar, one = res
    for k in ("n_refined_tiles", "arg_i", "arg_e", "arg_o", "ln_z", "max_lnl_ml", "n_eff", "n_marginalised"):
        assert wide[k] == one[k], k
    assert wide["n_refined_tiles"] == nar["n_refined_tiles"]
    assert (wide["arg_i"], wide["arg_e"], wide["arg_o"]) == (nar["arg_i"], nar["arg_e"], nar["arg_o"])
    assert wide["ln_z"] == pytest.approx(nar["ln_z"], abs=1e-9)
    assert wide["max_lnl_ml"] == nar["max_lnl_ml"]
    if (i1 - i0) * E > 300000:
        bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
        try:
            ref = run(dp, ctx, wl, "fp32", bid=bid, i0=i0, i1=i1, cut=20.0, flags=0)["ev"]
        finally:
            dp.dotpe_bank_release(ctx, bid)
        assert abs(wide["ln_z"] - ref["ln_z"]) <= 1e-2
        assert wide["max_lnl_ml"] == pytest.approx(ref["max_lnl_ml"], abs=1e-3)
        assert (wide["arg_i"], wide["arg_e"], wide["arg_o"]) == (ref["arg_i"], ref["arg_e"], ref["arg_o"])
        return
    P = oracle.OracleProblem(wl.bank, wl.ext, wl.event, i_slice=slice(i0, i1))
    gcut, thr = P.eval_grid(20.0)
    guncut, _ = P.eval_grid(0.0)
    lo, hi = P.evidence(gcut)["ln_z"], P.evidence(guncut)["ln_z"]
    assert lo - 1e-2 <= wide["ln_z"] <= hi + 1e-2
    assert wide["max_lnl_ml"] == pytest.approx(float(guncut["lnl_ml_max"].max()), abs=1e-3)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_bank_shards_merge_to_one_pass(dpx, precision):
    """A bank-sharded event on one GPU: the slice's rows in two shards (each an
    event of its own), merged by dotpe_evidence_merge, give the one-pass
    event's ln Z, N_eff, N_eff,int, N_eff,ext, per-sample marginals and maximum
    (the shards' tiles are the one-pass event's, so the FP32 tile partials are
    the same; the per-sample marginals arrive as float32)."""
    dp, ctx = dpx
    wl = synth.make_workload(n_int=600, n_ext=90, n_det=3, n_modes=4, n_bins=128, snr=14.0, seed=71,
                             ln_w="random")
    bid = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        one = run(dp, ctx, wl, precision, bid=bid, i0=0, i1=600, flags=0)
        shards = []
        for a, b in ((0, 256), (256, 600)):
            got = run(dp, ctx, wl, precision, bid=bid, i0=a, i1=b, flags=0)
            shards.append((got["ev"], b - a, got["col"].astype(np.float64)))
    finally:
        dp.dotpe_bank_release(ctx, bid)
    merged, lpe = dp.dotpe_evidence_merge(shards, wl.event.n_phi)
    ev = one["ev"]
    assert merged["ln_z"] == pytest.approx(ev["ln_z"], abs=1e-9)
    assert merged["n_eff"] == pytest.approx(ev["n_eff"], rel=1e-9)
    assert merged["n_eff_int"] == pytest.approx(ev["n_eff_int"], rel=1e-9)
    assert merged["n_eff_ext"] == pytest.approx(ev["n_eff_ext"], rel=1e-5)
    np.testing.assert_allclose(lpe, one["col"].astype(np.float64), rtol=0, atol=1e-5)
    assert merged["max_lnl_ml"] == ev["max_lnl_ml"]
    assert (merged["arg_i"], merged["arg_e"], merged["arg_o"]) == (ev["arg_i"], ev["arg_e"], ev["arg_o"])
    assert merged["n_marginalised"] == ev["n_marginalised"] and merged["n_pairs"] == ev["n_pairs"]


def test_gemm_only_diagnostic_runs(dpx):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=1024, n_ext=256, n_det=3, n_modes=4, n_bins=256, seed=2)
    for precision in ("bf16", "bf16x3", "fp32"):
        got = run(dp, ctx, wl, precision, flags=dp.DOTPE_FLAG_GEMM_ONLY)
        assert got["stats"]["fused_ms"] > 0
