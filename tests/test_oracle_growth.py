"""Growth rates of the FP64 oracle against the exact solution of Eq. 5 (CPU only, ~40 s).

Cold pair beam in the paper's 2D3V geometry with one seeded transverse mode (k = 2, Gamma =
4e-3).  The local rate Gamma^st = d_tau ln|psi| (blazar paragraph of the paper) is fitted over
Gamma tau in [2, 5] at xi = 2 (spatiotemporal filamentation, near the front) and xi = 20
(spatiotemporal oblique mode), and must match the same fit of the exact series within 3%.
"""
import math

import numpy as np

from oracle import linear_theory as lt
from oracle import qspic
from paper_2607_24214_b300 import config, inputs


def test_growth_rates_match_eq5_series():
    p = config.v_pair_single_mode()
    my = p.modes[0].my
    k = 2 * math.pi * my / p.Ly
    G = lt.growth_rate(k, p.species)
    assert abs(G - 4e-3) < 1e-6
    beams = inputs.all_beams(p)
    amps = []
    for n in range(p.steps + 1):
        slab, d = qspic.plasma_sweep(p, qspic.beam_sources(p, beams))
        Wy = np.fft.fft(slab[:, 1, :, 0], axis=1)[:, my]          # W_y = -d_y psi
        amps.append(np.abs(Wy) / k)
        if n < p.steps:
            qspic.beam_push(p, beams, slab)
    amps = np.array(amps)
    taus = np.arange(p.steps + 1) * p.dt
    sel = (G * taus >= 2.0) & (G * taus <= 5.0)
    for xi in (2.0, 20.0):
        j = int(round(xi / p.dxi))
        ex = np.array([abs(lt.psi_series(xi, G * t, 1.0, k)) for t in taus[sel]])
        rate_sim = np.polyfit(taus[sel], np.log(amps[sel, j]), 1)[0]
        rate_ex = np.polyfit(taus[sel], np.log(ex), 1)[0]
        assert abs(rate_sim / rate_ex - 1) < 0.03, (xi, rate_sim / G, rate_ex / G)
        # OTSI dominates deep in the beam, CFI grows slower near the front (Eqs. 6-7)
    j2, j20 = int(round(2 / p.dxi)), int(round(20 / p.dxi))
    assert amps[-1, j20] / amps[0, j20] > amps[-1, j2] / amps[0, j2]
