"""Batched launches, continuous batching, graph replay and the band autotuner.

Every result is compared with the one the same event gets when submitted
alone.  The comparisons are bitwise: a batch evaluates the same tiles with the
same code and reduces each event's partials in a fixed order.  Runs without
the ML cut (or with it in mixed precision, whose refinement threshold is
frozen) are deterministic; a running-maximum cut is not compared bitwise.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

KEYS = ("ln_z", "n_eff", "n_eff_int", "n_eff_ext", "max_lnl_ml", "arg_i", "arg_e", "arg_o", "n_marginalised",
        "lnl_ml_threshold", "n_refined_tiles")


@pytest.fixture(scope="module")
def mix():
    import __graft_entry__ as ge
    ge.build()
    import paper_2507_16022_gb300 as dp
    wl = synth.make_workload(n_int=6144, n_ext=64, n_det=3, n_modes=4, n_bins=256, snr=12.0, seed=41,
                             ln_w="random")
    rng = np.random.default_rng(17)
    specs = []
    # uneven slices, extrinsic counts (ragged tiles), detector counts and SNR
    for k, (E, D, snr, a, b) in enumerate([(512, 3, 10.0, 0, 6144), (300, 2, 25.0, 128, 4000),
                                           (1024, 3, 15.0, 2048, 2900), (96, 2, 40.0, 0, 6144),
                                           (700, 3, 8.0, 1000, 6100)]):
        ext = synth.make_extrinsic(np.random.default_rng(200 + k), E, D, wl.bank, ln_w="random")
        ev = synth.make_event(rng, wl.bank, ext, D, snr=snr, inj_i=int(rng.integers(a, b)))
        specs.append(dict(i0=a, i1=b, psd=ev.psd, data=ev.data, t=ext.t, R=ext.R, ln_w_ext=ext.ln_w,
                          n_phi=32, u_min=ev.u_min))
    return dp, wl, specs


def load(dp, ctx, wl):
    return dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)


def alone(dp, ctx, bid, specs, precision, cut):
    out = []
    for sp in specs:
        eid = dp.dotpe_event_submit(ctx, bid, precision=precision, cut_delta=cut, **sp)
        dp.dotpe_event_wait(ctx, eid, 120.0)
        out.append(dp.dotpe_evidence(ctx, eid))
        dp.dotpe_event_release(ctx, eid)
    return out


def collect(dp, ctx, ids):
    out = []
    for eid in ids:
        dp.dotpe_event_wait(ctx, eid, 120.0)
        out.append(dp.dotpe_evidence(ctx, eid))
        dp.dotpe_event_release(ctx, eid)
    return out


def same(a_list, b_list):
    for a, b in zip(a_list, b_list):
        for k in KEYS:
            assert a[k] == b[k], (k, a[k], b[k])


@pytest.mark.parametrize("precision,cut", [("bf16x3", 0.0), ("mixed", 20.0), ("mixed", 0.0), ("fp16", 0.0),
                                           ("fp32", 0.0)])
def test_batch_equals_alone(mix, precision, cut):
    dp, wl, specs = mix
    ctx = dp.dotpe_create(0)
    try:
        bid = load(dp, ctx, wl)
        ref = alone(dp, ctx, bid, specs, precision, cut)
        for rep in range(2):  # the second batch replays the updated executable graph
            ids = dp.dotpe_batch_submit(ctx, [dict(bank_id=bid, precision=precision, cut_delta=cut, **sp)
                                              for sp in specs])
            same(ref, collect(dp, ctx, ids))
        dp.dotpe_bank_release(ctx, bid)
    finally:
        dp.dotpe_destroy(ctx)


def test_batch_without_graphs(mix):
    dp, wl, specs = mix
    ctx = dp.dotpe_create(0, flags=dp.DOTPE_CONFIG_NO_GRAPHS)
    try:
        bid = load(dp, ctx, wl)
        ref = alone(dp, ctx, bid, specs, "mixed", 20.0)
        ids = dp.dotpe_batch_submit(ctx, [dict(bank_id=bid, precision="mixed", cut_delta=20.0, **sp)
                                          for sp in specs])
        same(ref, collect(dp, ctx, ids))
        dp.dotpe_bank_release(ctx, bid)
    finally:
        dp.dotpe_destroy(ctx)


def test_continuous_batching(mix):
    """One slot: the first event runs alone; the events that arrive meanwhile
    queue and are admitted together as one batch when the slot frees."""
    import torch
    dp, wl, specs = mix
    ctx = dp.dotpe_create(0, n_slots=1, max_batch=8)
    try:
        bid = load(dp, ctx, wl)
        ref = alone(dp, ctx, bid, specs, "mixed", 20.0)
        # the first event's inputs wait behind ~50 ms of work on the caller's stream,
        # so the others surely arrive while it holds the slot
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            torch.cuda._sleep(100_000_000)
        ids = [dp.dotpe_event_submit(ctx, bid, precision="mixed", cut_delta=20.0, stream=s, **specs[0])]
        ids += [dp.dotpe_event_submit(ctx, bid, precision="mixed", cut_delta=20.0, **sp) for sp in specs[1:]]
        for eid in ids:
            dp.dotpe_event_wait(ctx, eid, 120.0)
        admits = [dp.dotpe_event_poll(ctx, eid)[1]["t_admit_ns"] for eid in ids]
        same(ref, collect(dp, ctx, ids))
        # the events that queued behind the first were admitted together, after it
        assert len(set(admits[1:])) == 1 and admits[1] > admits[0]
    finally:
        dp.dotpe_destroy(ctx)


def test_batch_admission_errors(mix):
    dp, wl, specs = mix
    ctx = dp.dotpe_create(0)
    try:
        bid = load(dp, ctx, wl)
        mixed_prec = [dict(bank_id=bid, precision=p, **specs[0]) for p in ("mixed", "bf16x3")]
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_batch_submit(ctx, mixed_prec)
        assert ei.value.status == dp.DOTPE_E_INVALID
        bad = [dict(bank_id=bid, precision="mixed", **sp) for sp in specs[:2]]
        bad[1] = dict(bad[1], n_phi=0)
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_batch_submit(ctx, bad)
        assert ei.value.status == dp.DOTPE_E_INVALID
        # nothing of the refused batches stays queued: a good batch still runs
        ids = dp.dotpe_batch_submit(ctx, [dict(bank_id=bid, precision="mixed", **sp) for sp in specs[:2]])
        assert len(collect(dp, ctx, ids)) == 2
        dp.dotpe_bank_release(ctx, bid)
    finally:
        dp.dotpe_destroy(ctx)


def test_autotuned_band_gives_the_same_result(mix):
    """The autotuner changes only the order of the tiles (the L2 band width)."""
    dp, wl, specs = mix
    ref_ctx = dp.dotpe_create(0)
    ctx = dp.dotpe_create(0, flags=dp.DOTPE_CONFIG_AUTOTUNE)
    try:
        b0, b1 = load(dp, ref_ctx, wl), load(dp, ctx, wl)
        for precision, cut in (("bf16x3", 0.0), ("mixed", 20.0)):
            ref = alone(dp, ref_ctx, b0, specs, precision, cut)
            same(ref, alone(dp, ctx, b1, specs, precision, cut))   # tunes on first use of each shape
            same(ref, alone(dp, ctx, b1, specs, precision, cut))   # tuned widths from the cache
    finally:
        dp.dotpe_destroy(ctx)
        dp.dotpe_destroy(ref_ctx)
