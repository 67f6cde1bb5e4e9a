"""The saturation estimates and growth exponents used to read the nonlinear pair-beam run,
against the numbers the paper works out for its blazar run (alpha = 1e-10 per species,
gamma_b = 1e6, k_y = k_p; filamentation read at xi = 2 with omega_p tau_sat = 7e8,
oblique two-stream at xi = 30 with omega_p tau_sat = 5e8), and against the exponents'
own limits.  The paper rounds its results to one or two figures."""
import math

import numpy as np
import pytest

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


def _flat_top_bunch_wake(alpha, length, half_width=None):
    """On-axis E_z oscillation amplitude behind an electron bunch of density alpha, flat-top
    of length `length` from the front, in the FP64 oracle's QS-PIC (small alpha: the linear
    regime).  Without half_width the bunch fills the transverse box; with it the bunch is a
    slab |y - Ly/2| < half_width in the paper's 2D3V geometry (nx = 1)."""
    from oracle import qspic
    from paper_2607_24214_b300 import inputs
    dxi = 0.0625
    if half_width is None:
        p = config.Params(nx=4, ny=4, nxi=int(16 / dxi), Lx=1.0, Ly=1.0, Lxi=16.0, dt=1.0,
                          species=[config.Species(Z=-1, M=1, alpha=alpha, gamma_b=1e3,
                                                  xi_back=length)])
        slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, inputs.all_beams(p)))
        ez = d["ez0"]
    else:
        ny, Ly = 256, 25.6
        dy = Ly / ny
        p = config.Params(nx=1, ny=ny, nxi=int(12 / dxi), Lx=dy, Ly=Ly, Lxi=12.0, dt=1.0,
                          species=[config.Species(Z=-1, M=1, alpha=alpha, gamma_b=1e3)],
                          ppc_plasma_x=1, ppc_plasma_y=2)
        iy = np.arange(int(round((Ly / 2 - half_width) / dy)),
                       int(round((Ly / 2 + half_width) / dy)))
        ks = np.arange(int(round(length / dxi)))
        Y, XI = np.meshgrid(np.concatenate([(iy + 0.25) * dy, (iy + 0.75) * dy]),
                            np.concatenate([(ks + 0.25) * dxi, (ks + 0.75) * dxi]))
        n = Y.size
        b = dict(x=np.full(n, 0.5 * dy), y=Y.ravel(), xi=XI.ravel(), ux=np.zeros(n),
                 uy=np.zeros(n), uz=np.full(n, math.sqrt(1e6 - 1.0)),
                 w=np.full(n, alpha * dy * dy * dxi / 4))
        slab, _ = qspic.plasma_sweep(p, qspic.beam_sources(p, [b]))
        ez = slab[:, 2, int(round(Ly / 2 / dy)), 0]
    xs = np.arange(p.nxi + 1) * dxi
    return np.abs(ez[xs > length + 0.5]).max()


def test_filament_wake_estimate_against_the_qspic_response():
    """The filament wake estimate |2 rho_b sin(l/2)| (1 - exp(-w)) of the blazar paragraph
    against the oracle's plasma response to a flat-top bunch of length l (Eq. 1 with a
    step-on, step-off source): unbounded in the transverse plane (the first factor alone),
    and a slab of half-width w in the 2D geometry (the width factor); both within 1 %."""
    alpha = 1e-4
    for length in (5.0, 2.0):
        got = _flat_top_bunch_wake(alpha, length)
        assert abs(got / nl.ex_wake_amplitude(alpha, length, np.inf) - 1) < 0.01, length
    for w in (1.0, 0.5):
        got = _flat_top_bunch_wake(alpha, 5.0, half_width=w)
        assert abs(got / nl.ex_wake_amplitude(alpha, 5.0, w) - 1) < 0.01, w
    # the longitudinal spread the wakes build: |rho_b| tau
    assert nl.dpx_spread(-2e-10, 1e10) == pytest.approx(2.0)


def test_filament_sizes_of_synthetic_filaments():
    """filament_sizes on Gaussian filaments of known spacing, width and length (square and
    jittered lattices): spacing exact, width within 6 %, length within one slice."""
    rng = np.random.default_rng(0)
    n, h, dxi, nk = 64, 0.125, 0.125, 80
    X, Y = np.meshgrid(np.arange(n) * h, np.arange(n) * h)
    B = n * h
    for s, lam, length, jitter in ((0.25, 2.0, 5.0, 0.0), (0.4, 2.0, 3.0, 0.0),
                                   (0.3, 1.6, 6.0, 0.0), (0.3, 2.0, 5.0, 0.3)):
        f = np.zeros((n, n))
        for cx in np.arange(0.3, B, lam):
            for cy in np.arange(0.3, B, lam):
                jx, jy = rng.uniform(-jitter, jitter, 2)
                dx_ = np.mod(X - cx - jx + B / 2, B) - B / 2
                dy_ = np.mod(Y - cy - jy + B / 2, B) - B / 2
                f += np.exp(-(dx_ ** 2 + dy_ ** 2) / (2 * s * s))
        rho = np.array([f if (k + 0.5) * dxi < length else 0 * f for k in range(nk)])
        r = nl.filament_sizes(rho, h, h, dxi)
        assert r["spacing"] == pytest.approx(lam)
        assert abs(r["width"] / (2 * math.sqrt(2 * math.log(2)) * s) - 1) < 0.06, (s, r)
        assert abs(r["length"] - length) <= dxi, (length, r)
