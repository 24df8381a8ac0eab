"""Pins of the oracle's incoherent single-detector pre-selection (Sec. IV.D,
App. B) against what the mathematics fixes.

The single-detector maximum likelihood over the two polarisation amplitudes
is the squared length of the data's projection onto the plane the two
polarisation templates span (Eqs. x_ML, single_det_ML).  The pins compute that
projection by least squares on explicitly built whitened real vectors, use the
matched-filter closed form of a single mode (App. C's distance-optimised SNR
timeseries), a noiseless injection placed on the grid, invariances the
definition implies, and the chi-squared statistics of pure noise.
"""
import math

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def whiten(a, omega):
    """Real vector v(a) with v(a).v(b) = Re sum_b omega a b^*, the inner product of Eq. inner_product."""
    r = np.sqrt(omega)
    return np.concatenate([a.real * r, a.imag * r])


def projection_ml(vd, cols):
    """1/2 |P d|^2 with P the orthogonal projector onto span(cols), by least squares."""
    A = np.stack(cols, axis=1)
    x, *_ = np.linalg.lstsq(A, vd, rcond=1e-12)
    res = vd - A @ x
    return 0.5 * (vd @ vd - res @ res)


def tiny_problem(seed, I=3, D=2, M=3, B=24, NT=5, mode_m=(1, 2, 3)):
    rng = np.random.default_rng(seed)
    f = np.linspace(20.0, 300.0, B)
    w = np.full(B, f[1] - f[0])
    psd = rng.uniform(0.5, 2.0, (D, B))
    h = rng.standard_normal((I, M, B)) + 1j * rng.standard_normal((I, M, B))
    pol = rng.standard_normal((I, M, 2)) + 1j * rng.standard_normal((I, M, 2))
    data = rng.standard_normal((D, B)) + 1j * rng.standard_normal((D, B))
    t_grid = rng.uniform(-0.01, 0.01, (D, NT))
    return dict(f=f, w=w, mode_m=np.array(mode_m[:M]), h=h, pol=pol, psd=psd, data=data, t_grid=t_grid)


def templates(p, i, k, o, t, n_phi):
    """h_{i k o t p}(f_b) of Eq. dh_itop, built directly: sum_m K_{imp} h_{im} e^{i m phi_o} e^{-2 pi i f t}."""
    phi = 2.0 * np.pi * o / n_phi
    shift = np.exp(-2j * np.pi * p["f"] * p["t_grid"][k, t])
    out = []
    for q in range(2):
        s = np.zeros_like(p["f"], dtype=np.complex128)
        for m in range(p["h"].shape[1]):
            s += p["pol"][i, m, q] * p["h"][i, m] * np.exp(1j * p["mode_m"][m] * phi)
        out.append(s * shift)
    return out


# ---------------------------------------------------------------------------
# Eqs. x_ML, single_det_ML on explicit vectors
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["generic", "parallel", "zero_cross", "zero_both", "orthogonal"])
def test_quad_ml_is_the_projection(orc, case):
    rng = np.random.default_rng(hash(case) % 2 ** 32)
    for _ in range(20):
        d = rng.standard_normal(12)
        hp = rng.standard_normal(12)
        hx = rng.standard_normal(12)
        if case == "parallel":
            hx = -2.5 * hp
        elif case == "zero_cross":
            hx = np.zeros(12)
        elif case == "zero_both":
            hp = np.zeros(12)
            hx = np.zeros(12)
        elif case == "orthogonal":
            hx = hx - (hx @ hp) / (hp @ hp) * hp
        got = orc.quad_ml(d @ hp, d @ hx, hp @ hp, hp @ hx, hx @ hx)
        want = projection_ml(d, [hp, hx]) if case != "zero_both" else 0.0
        assert got == pytest.approx(want, rel=1e-10, abs=1e-12)


# ---------------------------------------------------------------------------
# Eq. dh_itop + Eq. single_det_ML: the grid against a projection of explicit templates
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [1, 2])
def test_presel_grid_equals_projection_of_built_templates(orc, seed):
    p = tiny_problem(seed)
    n_phi = 6
    P = orc.PreselProblem(n_phi=n_phi, **p)
    I, M, B = p["h"].shape
    D, NT = p["t_grid"].shape
    for i in range(I):
        for k in range(D):
            g = P.grid(i, k)
            omega = 4.0 * p["w"] / p["psd"][k]
            vd = whiten(p["data"][k], omega)
            for o in range(n_phi):
                for t in range(NT):
                    hp, hx = templates(p, i, k, o, t, n_phi)
                    want = projection_ml(vd, [whiten(hp, omega), whiten(hx, omega)])
                    assert g[o, t] == pytest.approx(want, rel=1e-10), (i, k, o, t)


def test_single_mode_is_the_matched_filter_snr(orc):
    """One mode with independent (over the reals) K+, Kx: the two templates span
    the complex line of h, so ln L^ML = |<d|h>_C|^2 / (2 <h|h>) at every phase
    (App. C's distance-optimised rho_k^2(t))."""
    p = tiny_problem(5, I=2, D=2, M=1, mode_m=(2,))
    n_phi = 8
    P = orc.PreselProblem(n_phi=n_phi, **p)
    for i in range(2):
        for k in range(2):
            omega = 4.0 * p["w"] / p["psd"][k]
            hh = np.sum(omega * np.abs(p["h"][i, 0]) ** 2)
            g = P.grid(i, k)
            for t in range(p["t_grid"].shape[1]):
                shift = np.exp(-2j * np.pi * p["f"] * p["t_grid"][k, t])
                z = np.sum(omega * np.conj(p["data"][k]) * shift * p["h"][i, 0])
                np.testing.assert_allclose(g[:, t], abs(z) ** 2 / (2 * hh), rtol=1e-10)


def test_noiseless_injection_on_the_grid(orc):
    """d_k = x+ h+ + xx hx of row i* at (o*, t*): that point reaches <d_k|d_k>/2,
    nothing exceeds it (a projection never lengthens), and the row is the
    maximum of ln L^inco.ML."""
    p = tiny_problem(7, I=4, D=3, M=4, B=40, NT=6, mode_m=(1, 2, 3, 4))
    n_phi = 8
    i_star, o_star = 2, 3
    rng = np.random.default_rng(70)
    half_dd = []
    for k in range(3):
        t_star = k + 1
        hp, hx = templates(p, i_star, k, o_star, t_star, n_phi)
        p["data"][k] = rng.normal() * hp + rng.normal() * hx
        omega = 4.0 * p["w"] / p["psd"][k]
        half_dd.append(0.5 * np.sum(omega * np.abs(p["data"][k]) ** 2))
    P = orc.PreselProblem(n_phi=n_phi, **p)
    r = P.run(delta=20.0)
    for k in range(3):
        assert r["ml"][i_star, k] == pytest.approx(half_dd[k], rel=1e-10)
        assert tuple(r["arg_ot"][i_star, k]) == (o_star, k + 1)
        assert np.all(r["ml"][:, k] <= half_dd[k] * (1 + 1e-12))
    assert r["arg_i"] == i_star
    assert r["lnl_inco"][i_star] == pytest.approx(sum(half_dd), rel=1e-10)


def test_real_mixing_of_the_polarisations_changes_nothing(orc):
    """x_p are free real amplitudes: any real invertible recombination of the two
    polarisation templates, and any real rescaling of a row, spans the same plane."""
    p = tiny_problem(11)
    n_phi = 6
    base = orc.PreselProblem(n_phi=n_phi, **p)
    rng = np.random.default_rng(12)
    q = dict(p)
    A = rng.standard_normal((p["h"].shape[0], 2, 2))
    q["pol"] = np.einsum("imp,ipq->imq", p["pol"], A)
    q["h"] = p["h"] * rng.uniform(0.2, 5.0, (p["h"].shape[0], 1, 1))
    mixed = orc.PreselProblem(n_phi=n_phi, **q)
    for i in range(p["h"].shape[0]):
        for k in range(p["t_grid"].shape[0]):
            np.testing.assert_allclose(mixed.grid(i, k), base.grid(i, k), rtol=1e-9)


def test_edge_on_row_takes_the_rank_one_limit(orc):
    """cos(iota) = 0: every Kx vanishes, <h|h> has rank one, and the maximum is
    the projection onto h+ alone."""
    wl = synth.make_workload(n_int=2, n_ext=2, n_det=2, n_modes=4, n_bins=32, seed=3)
    pol = synth.row_polarisation_factors(wl.bank, np.array([0.0, 0.4]))
    pol[0, :, 1] = 0.0  # exactly edge-on (the closed forms leave ~1e-17)
    t_grid = np.array([[-1e-3, 0.0, 2e-3]] * 2)
    P = orc.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, pol, wl.event.psd,
                          wl.event.data, t_grid, n_phi=4)
    p = dict(f=wl.bank.f, h=wl.bank.h, pol=pol, mode_m=wl.bank.mode_m, t_grid=t_grid)
    for k in range(2):
        g = P.grid(0, k)
        omega = 4.0 * wl.bank.w / wl.event.psd[k]
        vd = whiten(wl.event.data[k], omega)
        for o in range(4):
            for t in range(3):
                hp, _ = templates(p, 0, k, o, t, 4)
                assert g[o, t] == pytest.approx(projection_ml(vd, [whiten(hp, omega)]), rel=1e-10)


def test_selection_window_and_row_maxima(orc):
    wl = synth.make_workload(n_int=24, n_ext=2, n_det=3, n_modes=4, n_bins=64, seed=21, snr=12.0)
    ps = synth.make_presel_inputs(wl, n_t=16, dt=2e-3)
    P = orc.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, ps.pol, wl.event.psd,
                          wl.event.data, ps.t_grid, n_phi=8)
    for delta in (5.0, 20.0):
        r = P.run(delta=delta)
        assert r["threshold"] == pytest.approx(r["lnl_inco"].max() - delta, abs=0)
        assert r["arg_i"] == int(np.argmax(r["lnl_inco"]))
        np.testing.assert_array_equal(r["keep"], r["lnl_inco"] >= r["lnl_inco"].max() - delta)
        np.testing.assert_allclose(r["lnl_inco"], r["ml"].sum(axis=1), rtol=1e-14)
    for i in (0, 7, wl.event.injection["i"]):
        for k in range(3):
            g = P.grid(i, k)
            assert r["ml"][i, k] == g.max()
            o, t = r["arg_ot"][i, k]
            assert g[o, t] == g.max()


def test_noise_only_projection_is_chi_squared_with_two_dof(orc):
    """White Gaussian noise with Re<n|h> ~ N(0, <h|h>): 2 ln L^ML at a fixed
    (i, k, o, t) is chi^2 with 2 degrees of freedom (mean 2, variance 4)."""
    wl = synth.make_workload(n_int=1, n_ext=1, n_det=1, n_modes=4, n_bins=48, seed=4)
    ps = synth.make_presel_inputs(wl, n_t=2, dt=1e-3, seed=5)
    rng = np.random.default_rng(99)
    sigma = np.sqrt(wl.event.psd / (4.0 * wl.bank.w[None, :]))
    vals = []
    for _ in range(1500):
        n = sigma * (rng.standard_normal(sigma.shape) + 1j * rng.standard_normal(sigma.shape))
        P = orc.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, ps.pol, wl.event.psd,
                              n, ps.t_grid, n_phi=4)
        vals.append(2.0 * P.grid(0, 0)[1, 0])
    vals = np.array(vals)
    # mean 2 +- 5 sigma (sigma = 2/sqrt(1500)); exponential tail P(chi2_2 > 6) = e^-3
    assert abs(vals.mean() - 2.0) < 5 * 2.0 / math.sqrt(len(vals))
    assert abs(np.mean(vals > 6.0) - math.exp(-3.0)) < 5 * math.sqrt(math.exp(-3) / len(vals))


# ---------------------------------------------------------------------------
# polarisation-resolved (precessing) bank: h_{i m p} read directly
# ---------------------------------------------------------------------------
def pol_templates(p, hpol, i, k, o, t, n_phi):
    """h_{i k o t p}(f_b) = sum_m h_{imp} e^{i m phi_o} e^{-2 pi i f t}, built directly."""
    phi = 2.0 * np.pi * o / n_phi
    shift = np.exp(-2j * np.pi * p["f"] * p["t_grid"][k, t])
    return [sum(hpol[i, m, q] * np.exp(1j * p["mode_m"][m] * phi) for m in range(hpol.shape[1])) * shift
            for q in range(2)]


@pytest.mark.parametrize("seed", [3, 4])
def test_polarisation_resolved_grid_equals_projection(orc, seed):
    """Random independent + and x components per mode (no common factor):
    the grid equals the projection onto the two built templates."""
    p = tiny_problem(seed)
    rng = np.random.default_rng(seed + 100)
    I, M, B = p["h"].shape
    hpol = rng.standard_normal((I, M, 2, B)) + 1j * rng.standard_normal((I, M, 2, B))
    n_phi = 5
    q = dict(p, h=hpol, pol=None)
    P = orc.PreselProblem(n_phi=n_phi, **q)
    D, NT = p["t_grid"].shape
    for i in range(I):
        for k in range(D):
            g = P.grid(i, k)
            omega = 4.0 * p["w"] / p["psd"][k]
            vd = whiten(p["data"][k], omega)
            for o in range(n_phi):
                for t in range(NT):
                    hp, hx = pol_templates(p, hpol, i, k, o, t, n_phi)
                    want = projection_ml(vd, [whiten(hp, omega), whiten(hx, omega)])
                    assert g[o, t] == pytest.approx(want, rel=1e-10), (i, k, o, t)


def test_polarisation_resolved_with_factors_is_the_mode_bank(orc):
    """h_{imp} = K_{imp} h_{im}: the pre-selection of the polarisation-resolved
    bank equals that of the mode bank with the factors (rows, maxima, kept set)."""
    wl = synth.make_workload(n_int=40, n_ext=4, n_det=3, n_modes=4, n_bins=64, seed=21)
    ps = synth.make_presel_inputs(wl, n_t=16, dt=5e-4, seed=22)
    hpol = wl.bank.h[:, :, None, :] * ps.pol[:, :, :, None]
    a = orc.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, wl.bank.h, ps.pol, wl.event.psd,
                          wl.event.data, ps.t_grid, n_phi=8).run(delta=20.0)
    b = orc.PreselProblem(wl.bank.f, wl.bank.w, wl.bank.mode_m, hpol, None, wl.event.psd,
                          wl.event.data, ps.t_grid, n_phi=8).run(delta=20.0)
    np.testing.assert_allclose(b["ml"], a["ml"], rtol=1e-11, atol=1e-11)
    np.testing.assert_array_equal(b["keep"], a["keep"])
