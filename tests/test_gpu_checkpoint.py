"""Checkpoint / resume of resident banks (dotpe_bank_save, dotpe_bank_open).

* A bank written to a file and opened again gives, event by event, the same
  per-pair values bit for bit (FP32, split fp16 and the pre-selection), for a
  mode bank with polarisation factors and ln w_int and for a
  polarisation-resolved bank.
* A damaged file is refused: a flipped payload byte (checksum), a flipped
  header byte (a mode number, the operand scale, the polarisation count: the
  checksum covers the header too, and the header's ranges are checked), a
  truncated payload, a wrong magic, a missing file.
"""
import struct

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


def lnl(dp, ctx, bid, wl, I, precision, F=None):
    eid = dp.dotpe_event_submit(ctx, bid, 0, I, wl.event.psd, wl.event.data, wl.ext.t,
                                None if F is not None else wl.ext.R, wl.ext.ln_w, n_phi=wl.event.n_phi,
                                u_min=wl.event.u_min, cut_delta=0.0, precision=precision,
                                flags=dp.DOTPE_FLAG_STORE_LNL, F=F)
    dp.dotpe_event_wait(ctx, eid, 120.0)
    E = wl.ext.t.shape[0]
    out = (dp.dotpe_lnl_blocks(ctx, eid, 0, I, 0, E), dp.dotpe_evidence(ctx, eid)["ln_z"])
    dp.dotpe_event_release(ctx, eid)
    return out


@pytest.mark.parametrize("kind", ["modes", "precessing"])
def test_saved_bank_gives_the_same_values(dpx, tmp_path, kind):
    dp, ctx = dpx
    if kind == "modes":
        wl = synth.make_workload(n_int=700, n_ext=100, n_det=3, n_modes=4, n_bins=256, seed=111, snr=14.0,
                                 ln_w="random")
        ps = synth.make_presel_inputs(wl, n_t=40, dt=1e-3, seed=112)
        pol, F = ps.pol, None
    else:
        wl = synth.make_precessing_workload(500, 90, 3, 4, 200, snr=14.0, seed=113, ln_w="random")
        pol, F = None, wl.ext.F
    I = wl.bank.h.shape[0]
    path = tmp_path / f"{kind}.bank"
    a = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w, pol=pol)
    b = None
    try:
        dp.dotpe_bank_save(ctx, a, path)
        b = dp.dotpe_bank_open(ctx, path)
        for precision in ("fp32", "fp16x3"):
            la, za = lnl(dp, ctx, a, wl, I, precision, F)
            lb, zb = lnl(dp, ctx, b, wl, I, precision, F)
            np.testing.assert_array_equal(lb, la)
            assert zb == za
        if kind == "modes":
            ra = dp.dotpe_preselect(ctx, a, 0, I, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16)
            rb = dp.dotpe_preselect(ctx, b, 0, I, wl.event.psd, wl.event.data, ps.t_grid, n_phi=16)
            np.testing.assert_array_equal(rb["lnl_ml"], ra["lnl_ml"])
    finally:
        dp.dotpe_bank_release(ctx, a)
        if b is not None:
            dp.dotpe_bank_release(ctx, b)


def test_damaged_files_are_refused(dpx, tmp_path):
    dp, ctx = dpx
    wl = synth.make_workload(n_int=200, n_ext=8, n_det=2, n_modes=2, n_bins=64, seed=114)
    path = tmp_path / "ok.bank"
    a = dp.dotpe_bank_load(ctx, wl.bank.h, wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.ln_w)
    try:
        dp.dotpe_bank_save(ctx, a, path)
    finally:
        dp.dotpe_bank_release(ctx, a)
    raw = bytearray(path.read_bytes())

    def flip(off, mask):
        return raw[:off] + bytes([raw[off] ^ mask]) + raw[off + 1:]

    # header: magic[8], version, n_pol (u32), n_int (i64), n_modes, n_bins, kpad,
    # has_lw, has_pol (i32), mode_m[4] (i32) at byte 44, a_scale (f32) at 60
    assert struct.unpack_from("<i", raw, 44)[0] == int(wl.bank.mode_m[0]) == 2
    damaged = {
        "flipped": flip(len(raw) - 100, 0x10),
        # m = 2 -> 1: still increasing and in 1..4, so only the checksum refuses it
        "mode_m in range": flip(44, int(wl.bank.mode_m[0]) ^ 1),
        "mode_m out of range": flip(44, 0x40),
        "second mode_m": flip(48, 0x04),
        "a_scale": flip(62, 0x01),
        "n_pol": flip(12, 0x02),
        "truncated": raw[:-1000],
        "magic": b"XXXXXXXX" + raw[8:],
    }
    for name, data in damaged.items():
        p = tmp_path / f"{name}.bank"
        p.write_bytes(bytes(data))
        with pytest.raises(dp.DotpeError) as ei:
            dp.dotpe_bank_open(ctx, p)
        assert ei.value.status == dp.DOTPE_E_INVALID, name
    with pytest.raises(dp.DotpeError) as ei:
        dp.dotpe_bank_open(ctx, tmp_path / "missing.bank")
    assert ei.value.status == dp.DOTPE_E_INVALID
