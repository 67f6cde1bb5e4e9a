"""Run parameters of the quasistatic PIC (QS-PIC) hot path and the named workloads.

Units are the paper's normalised ones (section "Quasistatic model"): time in 1/omega_p,
lengths in c/omega_p (k_p^-1), momenta in m_e c, densities in n_p, fields in
m_e c omega_p / e.  The propagation axis is z and xi = t - z is the comoving coordinate
of the QSA change of variables (the paper's (xi, tau) = (ct - x, t) with its x renamed z).
The transverse box is periodic (the QuaSSis paragraph: "transversely periodic boundary
conditions").  nx = 1 gives the paper's own 2D3V geometry (one transverse coordinate y).

This module holds plain data only: no arithmetic of the method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Tuple

MAX_SPECIES = 4
MAX_MODES = 16


@dataclass
class Species:
    """One beam species s: charge Z_s e, mass M_s m_e, density ratio alpha_s = n_bs/n_p,
    Lorentz factor gamma_b (model assumptions of the section "Quasistatic model")."""
    Z: float = -1.0
    M: float = 1.0
    alpha: float = 0.1
    gamma_b: float = 100.0
    gamma_spread_rel: float = 0.0   # std of gamma / gamma_b (Gaussian)
    uperp_spread: float = 0.0       # std of u_x, u_y in m_e c (Gaussian, thermal)
    noise_rel: float = 0.0          # std of the relative weight perturbation ("random weights")
    ppc_x: int = 2
    ppc_y: int = 2
    ppc_xi: int = 2
    xi_front: float = 0.0           # beam occupies [xi_front, xi_back)
    xi_back: float = -1.0           # < 0 means the back of the box, Lxi
    seeded: bool = False            # apply the seeded-mode list to this species' weights


@dataclass
class Mode:
    """Seeded transverse density mode: weight factor 1 + amplitude*cos(k.x + phase),
    k = (2 pi mx / Lx, 2 pi my / Ly)."""
    mx: int
    my: int
    amplitude: float
    phase: float = 0.0


@dataclass
class Params:
    nx: int
    ny: int
    nxi: int
    Lx: float
    Ly: float
    Lxi: float
    dt: float
    species: List[Species] = field(default_factory=list)
    modes: List[Mode] = field(default_factory=list)
    ppc_plasma_x: int = 2
    ppc_plasma_y: int = 2
    precision: str = "fp64"          # "fp64" or "mixed"
    n_pc_iter: int = 3
    pc_tol: float = 0.0              # > 0: solves per slice until the B_perp change < pc_tol
    psi_floor: float = 0.05
    seed: int = 0
    spin_limit: int = 1 << 26
    pipeline_depth: int = 1          # beam steps in flight per qsa_advance launch (1: none)
    rehome_frac: float = 0.0         # pipelined: re-home the beam when this fraction left its slots
    diag_modes: List[Tuple[int, int]] = field(default_factory=list)  # (mx, my) recorded per slice
    steps: int = 1                   # beam steps of the named workload (not part of the C struct)

    @property
    def dx(self):
        return self.Lx / self.nx

    @property
    def dy(self):
        return self.Ly / self.ny

    @property
    def dxi(self):
        return self.Lxi / self.nxi

    def with_(self, **kw) -> "Params":
        return replace(self, **kw)

    def plasma_per_slice(self) -> int:
        return self.nx * self.ny * self.ppc_plasma_x * self.ppc_plasma_y


DX_DEFAULT = 2.0 * math.pi / 32.0   # cell size used when a workload leaves the box unstated


def c1_fp64_electron_beam() -> Params:
    """Plain FP64 run: 32x32 transverse (box 2 pi), 64 slices over 8, 4 ppc plasma; electron
    beam alpha 0.1, gamma_b 100, thermal spread 1e-3, 8 ppc, 1e-3 weight noise; dt 5, 10 steps."""
    return Params(nx=32, ny=32, nxi=64, Lx=2 * math.pi, Ly=2 * math.pi, Lxi=8.0, dt=5.0,
                  species=[Species(Z=-1, M=1, alpha=0.1, gamma_b=100.0, uperp_spread=1e-3,
                                   noise_rel=1e-3)],
                  precision="fp64", steps=10)


def c2_mixed_electron_beam() -> Params:
    """Mixed-precision run: 256x256 transverse (box 16 pi), 1024 slices over 64, 4 ppc plasma;
    electron beam alpha 1e-2, gamma_b 1e3, spread 1e-4, 8 ppc, 1e-4 noise; dt 20, 200 steps."""
    L = 256 * DX_DEFAULT
    return Params(nx=256, ny=256, nxi=1024, Lx=L, Ly=L, Lxi=64.0, dt=20.0,
                  species=[Species(Z=-1, M=1, alpha=1e-2, gamma_b=1e3, uperp_spread=1e-4,
                                   noise_rel=1e-4)],
                  precision="mixed", steps=200)


def c3_pair_beam(ppc_xi: int = 1) -> Params:
    """Pair beam, 512x512 (box 32 pi), 2048 slices over 128; alpha 1e-4 per species, gamma_b
    1e4 with 1% energy spread; dt 200, 400 steps.  ppc_xi = 2 gives the workload's 2x2x2 = 8
    beam ppc per species (8.6e9 particles at 28 B: 275 GB on the device, which fits at
    pipeline depth 1 only); the default 2x2x1 = 4 leaves room for deeper pipelines and the
    diagnostics of the long run."""
    L = 512 * DX_DEFAULT
    sp = dict(alpha=1e-4, gamma_b=1e4, gamma_spread_rel=1e-2, noise_rel=1e-4, ppc_xi=ppc_xi)
    return Params(nx=512, ny=512, nxi=2048, Lx=L, Ly=L, Lxi=128.0, dt=200.0,
                  species=[Species(Z=-1, M=1, **sp), Species(Z=+1, M=1, **sp)],
                  precision="mixed", steps=400)


def pair_beam_filaments() -> Params:
    """Pair beam driven far into its nonlinear stage at moderate cost: 256 x 256 (box 16 pi),
    1024 slices over 64, electrons and positrons of alpha 1e-3 each, gamma_b 1e3, 1e-3 weight
    noise, 8 ppc; dt 20, 1000 steps.  Gamma = 1e-3 at k_y = k_p, so Gamma tau reaches 20: past
    saturation, into the stage of current filaments at the front whose wakes the blazar
    paragraph estimates.  Mixed precision."""
    L = 256 * DX_DEFAULT
    sp = dict(alpha=1e-3, gamma_b=1e3, noise_rel=1e-3)
    return Params(nx=256, ny=256, nxi=1024, Lx=L, Ly=L, Lxi=64.0, dt=20.0,
                  species=[Species(Z=-1, M=1, **sp), Species(Z=+1, M=1, **sp)],
                  precision="mixed", steps=1000)


def c4_parameter_scan(n: int = 64, seed: int = 0) -> List[Params]:
    """Batched scan: n independent instances, transverse grids drawn uniformly from
    {64, 96, 128, 192, 256}^2 (box N 2 pi / 32), 256 slices over 32, 4 ppc plasma; cold
    electron beam, alpha log-uniform in [1e-3, 1e-1], gamma_b log-uniform in [10, 1e3], 4 ppc
    (2x2x1), 1e-3 noise; dt = 0.1 / omega_b with omega_b = sqrt(alpha / gamma_b); 50 steps;
    mixed precision.  Instance i draws from Random(seed + i) and uses seed + i for its beam."""
    import random
    out = []
    for i in range(n):
        rng = random.Random(seed + i)
        N = rng.choice((64, 96, 128, 192, 256))
        alpha = 10 ** rng.uniform(-3, -1)
        gamma_b = 10 ** rng.uniform(1, 3)
        L = N * DX_DEFAULT
        out.append(Params(nx=N, ny=N, nxi=256, Lx=L, Ly=L, Lxi=32.0,
                          dt=0.1 / math.sqrt(alpha / gamma_b),
                          species=[Species(Z=-1, M=1, alpha=alpha, gamma_b=gamma_b, ppc_x=2,
                                           ppc_y=2, ppc_xi=1, noise_rel=1e-3)],
                          precision="mixed", steps=50, seed=seed + i))
    return out


def c5_seeded_modes(seed: int = 0) -> Params:
    """128x128 (box 8 pi), 256 slices over 32, electron beam alpha 1e-2, gamma_b 500, 8 ppc,
    16 seeded modes of amplitude 1e-3 (lowest |k| of the half plane, phases from the seed)."""
    import random
    L = 128 * DX_DEFAULT
    rng = random.Random(seed)
    ks = sorted({(mx, my) for mx in range(0, 4) for my in range(-3, 4)
                 if (mx > 0 or my > 0)}, key=lambda m: (m[0] ** 2 + m[1] ** 2, m))[:MAX_MODES]
    modes = [Mode(mx, my, 1e-3, rng.uniform(0, 2 * math.pi)) for mx, my in ks]
    return Params(nx=128, ny=128, nxi=256, Lx=L, Ly=L, Lxi=32.0, dt=20.0,
                  species=[Species(Z=-1, M=1, alpha=1e-2, gamma_b=500.0, seeded=True)],
                  modes=modes, precision="mixed", steps=50)


def v_pair_single_mode(ny: int = 128, Lxi: float = 21.0, dxi: float = 0.125, dt: float = 20.0,
                       steps: int = 62, my: int = 2, alpha: float = 1e-2, gamma_b: float = 1e3,
                       eps: float = 1e-7, precision: str = "fp64") -> Params:
    """Linear-growth validation in the paper's 2D3V geometry (nx = 1): cold pair beam, both
    species alpha each, electron weights seeded with one transverse mode k = 2 pi my / Ly
    (box 2 pi).  Defaults: k = 2, Gamma = 4e-3, Gamma tau_end = 4.96.  gamma_b = 1e3 keeps the
    slippage of the beam front, tau/(2 gamma_b^2), below 1e-3 (Eq. 5 assumes beta_b = 1);
    ny = 128 keeps the CIC smoothing of the mode below 0.1%; eps = 1e-7 keeps the seed
    linear through e^8 of growth.  Read at xi = 2 (filamentation, near the front) and xi = 20
    (oblique, deep in the beam)."""
    L = 2 * math.pi
    sp = dict(alpha=alpha, gamma_b=gamma_b, ppc_x=1, ppc_y=2, ppc_xi=2)
    return Params(nx=1, ny=ny, nxi=int(round(Lxi / dxi)), Lx=L / ny, Ly=L, Lxi=Lxi, dt=dt,
                  species=[Species(Z=-1, M=1, seeded=True, **sp), Species(Z=+1, M=1, **sp)],
                  modes=[Mode(0, my, eps, 0.0)], ppc_plasma_x=1, ppc_plasma_y=2,
                  precision=precision, steps=steps)
