"""Pins of the oracle's posterior resampling (Eq. posterior_element weights,
App. C distance draws).

* The distance draw inverts the conditional distance density, integrated and
  inverted independently here in d_L itself with scipy; the no-signal limit
  is the prior's closed form.
* The hierarchical draw (row, then extrinsic sample, then phase) reproduces
  the joint weights p_ie = w_i w_e sum_o Lbar_ieo computed directly from the
  per-pair grid, and the phase draw the per-phase weights of route O1.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize, stats

import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def d_quantile(dh, hh, u_min, q):
    """The q quantile of u = d0/d_L, returned as d_L/d0, by integrating
    pi(d) ~ d^2 exp(dh/d - hh/(2 d^2)) on (0, 1/u_min] in d (d0 = 1)."""
    dmax = 1.0 / u_min
    shift = dh * dh / (2 * hh) if dh > 0 else 0.0
    f = lambda d: d * d * math.exp(dh / d - 0.5 * hh / d ** 2 - shift)
    pts = [hh / dh] if (dh > 0 and hh / dh < dmax) else None
    tot = integrate.quad(f, 0, dmax, points=pts, epsabs=0, epsrel=1e-12, limit=400)[0]

    def g(x):
        p = [p for p in (pts or []) if p < x] or None
        return integrate.quad(f, 0, x, points=p, epsabs=0, epsrel=1e-12, limit=400)[0] / tot - (1 - q)
    # u <= u* <=> d >= d*: P(u <= u*) = 1 - CDF_d(d*)
    return optimize.brentq(g, 1e-9, dmax, xtol=1e-15)


@pytest.mark.parametrize("dh,hh,u_min,q", [(30.0, 4.0, 1.5, 0.3), (5.0, 1.0, 2.0, 0.7), (0.5, 0.2, 3.0, 0.5),
                                           (60.0, 16.0, 0.5, 0.95), (-2.0, 3.0, 1.0, 0.2), (12.0, 9.0, 2.5, 0.01)])
def test_distance_draw_inverts_the_conditional_density(orc, dh, hh, u_min, q):
    assert orc.dist_sample(dh, hh, u_min, q) == pytest.approx(d_quantile(dh, hh, u_min, q), rel=1e-9)


def test_distance_draw_without_signal_is_the_prior(orc):
    # pi(d) ~ d^2 on (0, dmax]: d/dmax = (1 - q)^(1/3) in the orientation u = d0/d
    for q in (0.0, 0.3, 0.9):
        assert orc.dist_sample(1.0, 0.0, 2.0, q) == pytest.approx((1 - q) ** (1 / 3) / 2.0, rel=1e-14)


def test_hierarchical_draw_reproduces_the_joint_weights(orc):
    wl = synth.make_workload(n_int=6, n_ext=5, n_det=2, n_modes=3, n_bins=48, seed=17, snr=6.0, n_phi=8,
                             ln_w="random")
    P = orc.OracleProblem(wl.bank, wl.ext, wl.event)
    grid, _ = P.eval_grid(0.0)
    ev = P.evidence(grid)
    rng = np.random.default_rng(18)
    n = 6000
    uni = rng.random((n, 4))
    i, e, o, d = orc.posterior_samples(P, grid, ev, uni)
    # joint weights straight from the grid: w_i w_e sum_o Lbar_ieo
    lp = wl.bank.ln_w[:, None] + wl.ext.ln_w[None, :] + grid["lnl_marg"]
    p = np.exp(lp - lp.max())
    p /= p.sum()
    counts = np.zeros_like(p)
    np.add.at(counts, (i, e), 1)
    keep = p * n >= 5
    chi2 = np.sum((counts[keep] - n * p[keep]) ** 2 / (n * p[keep]))
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4
    # phases of one pair: weights Lbar_ieo from route O1 (direct frequency sums)
    i0, e0 = np.unravel_index(np.argmax(p), p.shape)
    dh, hh = P.direct_phases(i0, e0)
    lo = np.array([orc.dist_marg(dh[q], hh[q], P.u_min) for q in range(P.n_phi)])
    po = np.exp(lo - lo.max())
    po /= po.sum()
    sel = (i == i0) & (e == e0)
    co = np.bincount(o[sel], minlength=P.n_phi)
    ok = po * sel.sum() >= 5
    chi2 = np.sum((co[ok] - sel.sum() * po[ok]) ** 2 / (sel.sum() * po[ok]))
    assert stats.chi2.sf(chi2, max(ok.sum() - 1, 1)) > 1e-4
    # distances of that pair and phase: Kolmogorov-Smirnov against the scipy CDF
    o0 = int(np.argmax(po))
    ds = d[sel & (o == o0)]
    if len(ds) >= 30:
        qs = np.linspace(0.02, 0.98, 25)
        dq = np.array([d_quantile(dh[o0], hh[o0], P.u_min, 1 - qq) for qq in qs])  # increasing in d
        emp = np.array([np.mean(ds <= x) for x in dq])
        assert np.max(np.abs(emp - qs)) < 1.7 / math.sqrt(len(ds))
