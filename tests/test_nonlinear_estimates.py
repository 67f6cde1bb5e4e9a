"""The saturation estimates and growth exponents used to read the nonlinear pair-beam run,
against the numbers the paper works out for its blazar run (alpha = 1e-10 per species,
gamma_b = 1e6, k_y = k_p; filamentation read at xi = 2 with omega_p tau_sat = 7e8,
oblique two-stream at xi = 30 with omega_p tau_sat = 5e8), and against the exponents'
own limits.  The paper rounds its results to one or two figures."""
import math

import numpy as np

from paper_2607_24214_b300 import config, nonlinear as nl


def pair(alpha, gamma_b):
    sp = dict(alpha=alpha, gamma_b=gamma_b, M=1.0)
    return [config.Species(Z=-1.0, **sp), config.Species(Z=1.0, **sp)]


def test_rate_at_ky_equal_kp_is_sqrt_alpha_over_gamma():
    # two species of omega_b^2 = alpha/gamma_b each, and k^2/(k^2+1) = 1/2 at k = 1
    G = nl.temporal_rate(1.0, pair(1e-10, 1e6))
    assert abs(G - 1e-8) <= 1e-22
    # large k: the unbounded rate (sum omega_b^2)^1/2
    assert abs(nl.temporal_rate(1e6, pair(1e-4, 1e4)) - math.sqrt(2e-8)) < 1e-16


def test_blazar_front_estimates():
    """Magnetic energy fraction ~2e-18 and momentum spread ~5e-3 at xi = 2, tau_sat = 7e8
    (the blazar paragraph after Eqs. 6-7)."""
    G = nl.temporal_rate(1.0, pair(1e-10, 1e6))
    eps = nl.eps_bz_sat(2.0, 7e8)
    assert abs(eps / 2e-18 - 1) < 0.05
    dp = nl.dpy_front(G, 2.0, 7e8, 1e6)
    assert abs(dp / 5e-3 - 1) < 0.1


def test_blazar_rear_estimates():
    """Electric energy fraction ~1.5e-16 and momentum spread ~0.016 at xi = 30,
    tau_sat = 5e8."""
    G = nl.temporal_rate(1.0, pair(1e-10, 1e6))
    eps = nl.eps_ey_sat(30.0, 5e8, 1e-10, 1e6)
    assert abs(eps / 1.5e-16 - 1) < 0.05
    dp = nl.dpy_rear(G, 30.0, 5e8, 1e6)
    assert abs(dp / 0.016 - 1) < 0.05


def test_trapping_balance_reproduces_the_estimates():
    """The estimates are the bounce frequency (k_y F / gamma_b)^1/2 set equal to the
    spatiotemporal rate, with F^2 = 4 alpha gamma_b eps: solve that balance directly."""
    a, g, ky, G = 1e-10, 1e6, 1.0, 1e-8
    for xi, ts in ((2.0, 7e8), (5.0, 1e9)):
        # front: k_y B / gamma_b = rate^2  =>  B = gamma_b rate^2 / k_y
        B = g * nl.rate_front(G, xi, ts) ** 2 / ky
        # the energy fraction uses the beam density; the front estimate is written with
        # the temporal rate folded in (Gamma^2 = alpha/gamma_b at k_y = k_p)
        assert abs(nl.fractional_energy(B * B, a, g) / nl.eps_bz_sat(xi, ts, ky) - 1) < 1e-12
    for xi, ts in ((30.0, 5e8), (20.0, 2e8)):
        E = g * nl.rate_rear(G, xi, ts) ** 2 / ky
        assert abs(nl.fractional_energy(E * E, a, g) / nl.eps_ey_sat(xi, ts, a, g, ky) - 1) < 1e-12


def test_exponents_and_rates_are_consistent():
    """The spatiotemporal rates are the tau-derivatives of the leading exponents."""
    G, tau, h = 3e-4, 2e4, 1.0
    for xi in (0.5, 2.0, 7.0):
        d = (nl.exponent_rear(G * (tau + h), xi) - nl.exponent_rear(G * (tau - h), xi)) / (2 * h)
        assert abs(d / nl.rate_rear(G, xi, tau) - 1) < 1e-6
        # the front exponent's leading term 2 (Gamma tau xi)^1/2
        lead = lambda gt: 2.0 * np.sqrt(gt * xi)
        d = (lead(G * (tau + h)) - lead(G * (tau - h))) / (2 * h)
        assert abs(d / nl.rate_front(G, xi, tau) - 1) < 1e-6
    # the two exponents meet the transition xi = 2 Gamma tau / sqrt 27 at the same order
    gt = 10.0
    xt = 2 * gt / math.sqrt(27.0)
    ratio = nl.exponent_front(gt, xt) / nl.exponent_rear(gt, xt)
    assert 0.8 < ratio < 1.3


def test_summary_reads_synthetic_growth():
    """`summary` on a record whose transverse fields grow exactly as Eq. 7 (front, B_perp) and
    Eq. 6 (downstream, E_perp): slopes 1 against the exponents, and at the end a growth rate
    equal to the spatiotemporal rate."""
    p = config.c3_pair_beam()
    G = nl.temporal_rate(1.0, p.species)
    tau = np.arange(1, 81) * 1000.0
    nseg = 64
    rs = np.full((tau.size, nseg, 6), 1e-12)
    xf, xr = 3.0, 21.0                       # centres of the segments [2, 4) and [20, 22)
    bf = 1e-9 * np.exp(nl.exponent_front(G * tau, xf))
    er = 1e-9 * np.exp(nl.exponent_rear(G * tau, xr))
    rs[:, 1, 3] = rs[:, 1, 4] = bf / np.sqrt(2.0)
    rs[:, 10, 0] = rs[:, 10, 1] = er / np.sqrt(2.0)
    rec = {"tau": tau, "rms_seg": rs, "energy": np.zeros((tau.size, 6)),
           "beam_rms_seg": np.zeros((tau.size, 2, nseg, 3)), "beam_lost": np.zeros(tau.size),
           "ms": np.ones(tau.size), "seg_width": np.float64(2.0)}
    s = nl.summary(rec, p)
    assert abs(s["front_Bperp"]["growth_vs_exponent"] - 1) < 1e-9
    assert abs(s["rear_Eperp"]["growth_vs_exponent"] - 1) < 1e-9
    # the last interval's mean rate against the rate at its midpoint (second-order close);
    # at the front the exponent's correction factor (1 - xi/(4 Gamma tau)) adds xi/(4 Gamma tau)
    # to the leading rate (Gamma xi/tau)^1/2
    tm = 0.5 * (tau[-1] + tau[-2])
    assert abs(s["front_Bperp"]["rate_ratio_end"] - (1 + xf / (4 * G * tm))) < 0.01
    assert abs(s["rear_Eperp"]["rate_ratio_end"] - 1) < 0.01
    assert abs(s["rear_Eperp"]["eps_end"] / nl.fractional_energy(er[-1] ** 2, 1e-4, 1e4) - 1) < 1e-12
